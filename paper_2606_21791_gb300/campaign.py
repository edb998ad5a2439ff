"""Resumable injection campaigns on the host.

A campaign's records depend only on each upset and the resident clean state,
so they can be kept on disk keyed by the upset's index in the list, and a
campaign of any length can stop (a crash, a pre-empted job) and continue where
it stopped with the same records an uninterrupted run gives.

Files of a campaign stored at `path` (a directory):
  records.npy    [n_upsets, K] gs_result records (numpy .npy, written in place)
  progress.json  {"done", "n", "K", "fingerprint", "setup"}: the number of
                 leading upsets whose records are on disk, a SHA-256 of the
                 upset list, and a digest of what else the records depend on
                 (scene, cameras, guard mode and box, word mask, tile shape:
                 `campaign_setup`); replaced atomically after the records of
                 each chunk are flushed, so "done" never counts a record that
                 is not on disk.

The chunk runner is the caller's: a function from a slice of the upset list to
its records, e.g. on the batched engine

    def run_chunk(fl):
        d, out = gs.to_device(fl), gs.device_bytes(len(fl) * K * gs.RESULT_DTYPE.itemsize)
        gs.gs_inject_and_render(scene, d, len(fl), 1, guard_mode, word_mask, out)
        torch.cuda.synchronize()
        return gs.from_device(out, gs.RESULT_DTYPE).reshape(len(fl), K)
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Callable, Optional

import numpy as np

from .gs import FLIP_DTYPE, RESULT_DTYPE


def flips_fingerprint(flips: np.ndarray) -> str:
    """SHA-256 of the upset list's bytes (prim, word, bit records in order)."""
    return hashlib.sha256(np.ascontiguousarray(flips).view(np.uint8).tobytes()).hexdigest()


def _digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).view(np.uint8).tobytes()).hexdigest()


def campaign_setup(planes, fmt: int, sh_degree: int, cams, guard_mode: int, word_mask: int,
                   box_lo=None, box_hi=None, tile=(16, 16)) -> dict:
    """What a campaign's records depend on besides the upsets, as a small
    JSON-able dict: the scene (format, SH degree, shape and a SHA-256 of its
    stored words), the cameras' bytes, the guard mode and word mask, the
    per-primitive box planes (if any) and the render tile shape."""
    planes = np.asarray(planes)
    return {"fmt": int(fmt), "sh_degree": int(sh_degree), "planes_shape": list(planes.shape),
            "planes_sha256": _digest(planes), "cams_sha256": _digest(np.asarray(cams)),
            "guard_mode": int(guard_mode), "word_mask": int(word_mask),
            "box_sha256": None if box_lo is None else _digest(np.concatenate(
                [np.asarray(box_lo).reshape(-1).view(np.uint8), np.asarray(box_hi).reshape(-1).view(np.uint8)])),
            "tile": [int(tile[0]), int(tile[1])]}


class ResumableCampaign:
    """The records of one campaign (upset list `flips`, `K` views, and
    `setup`, e.g. `campaign_setup(...)`) at `path`: created empty, or reopened
    where an earlier run stopped.  Reopening with a different upset list, view
    count or setup is refused (records of another scene, camera set, guard or
    tile shape would be mixed in silently otherwise)."""

    def __init__(self, path: str, flips: np.ndarray, K: int, setup: Optional[dict] = None):
        flips = np.ascontiguousarray(flips)
        if flips.dtype != FLIP_DTYPE or flips.ndim != 1:
            raise ValueError("flips must be a 1-D array of gs_flip records")
        if int(K) < 1:
            raise ValueError("K >= 1 views")
        self.path, self.flips, self.n, self.K = path, flips, len(flips), int(K)
        self.fingerprint = flips_fingerprint(flips)
        self.setup = json.loads(json.dumps(setup or {}))   # as stored
        os.makedirs(path, exist_ok=True)
        self.rec_path = os.path.join(path, "records.npy")
        self.prog_path = os.path.join(path, "progress.json")
        if os.path.exists(self.prog_path):
            with open(self.prog_path) as f:
                prog = json.load(f)
            if (prog.get("fingerprint") != self.fingerprint or prog.get("n") != self.n
                    or prog.get("K") != self.K):
                raise ValueError(f"another campaign (upset list or view count) is stored at {path}")
            if prog.get("setup", {}) != self.setup:
                raise ValueError(f"a campaign of another setup (scene, cameras, guard, tiles) is stored at {path}")
            self.records = np.lib.format.open_memmap(self.rec_path, mode="r+")
            if self.records.dtype != RESULT_DTYPE or self.records.shape != (self.n, self.K):
                raise ValueError(f"records at {path} do not match the campaign")
            self.done = int(prog["done"])
            if not 0 <= self.done <= self.n:
                raise ValueError(f"progress at {path} is out of range")
        else:
            self.records = np.lib.format.open_memmap(self.rec_path, mode="w+", dtype=RESULT_DTYPE,
                                                     shape=(self.n, self.K))
            self._commit(0)

    def _commit(self, done: int):
        self.records.flush()
        tmp = self.prog_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump({"done": int(done), "n": self.n, "K": self.K, "fingerprint": self.fingerprint,
                       "setup": self.setup}, f)
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, self.prog_path)
        self.done = int(done)

    def run(self, run_chunk: Callable[[np.ndarray], np.ndarray], chunk: int,
            max_chunks: Optional[int] = None) -> int:
        """Runs the upsets from `done` on, `chunk` at a time (at most
        `max_chunks` chunks), storing each chunk's records before counting it;
        returns the new `done`."""
        if int(chunk) < 1:
            raise ValueError("chunk >= 1")
        ran = 0
        while self.done < self.n and (max_chunks is None or ran < max_chunks):
            a = self.done
            b = min(self.n, a + int(chunk))
            out = np.asarray(run_chunk(self.flips[a:b]))
            if out.dtype != RESULT_DTYPE or out.shape != (b - a, self.K):
                raise ValueError(f"run_chunk returned {out.dtype} {out.shape}, want gs_result [{b - a}, {self.K}]")
            self.records[a:b] = out
            self._commit(b)
            ran += 1
        return self.done

    @property
    def complete(self) -> bool:
        return self.done == self.n
