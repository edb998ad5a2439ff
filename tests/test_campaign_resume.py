"""Resumable campaigns (host logic, no GPU): a run stopped part way -- by a
chunk limit or by an exception inside a chunk -- and resumed stores exactly
the records of an uninterrupted run; a different upset list or view count is
refused; a bad chunk result is rejected before anything is counted."""
import json
import os

import numpy as np
import pytest

from paper_2606_21791_gb300 import gs
from paper_2606_21791_gb300 import synth as S
from paper_2606_21791_gb300.campaign import ResumableCampaign, campaign_setup, flips_fingerprint

K = 3


def _records(fl):
    """A stand-in for the engine: records that depend only on each upset."""
    out = np.zeros((len(fl), K), dtype=gs.RESULT_DTYPE)
    for k in range(K):
        out["sse"][:, k] = fl["prim"] * 1e-3 + fl["word"] + k
        out["footprint"][:, k] = fl["bit"] + 10 * k
        out["maxabs"][:, k] = (fl["prim"] % 7) / 7.0
    return out


def _flips(n=1000, seed=5):
    return S.flips_stratified(n, 4000, 59, S.FP32, seed)


def test_stopped_and_resumed_equals_uninterrupted(tmp_path):
    fl = _flips()
    full = ResumableCampaign(str(tmp_path / "a"), fl, K)
    assert full.run(_records, 128) == len(fl) and full.complete

    c = ResumableCampaign(str(tmp_path / "b"), fl, K)
    assert c.run(_records, 128, max_chunks=3) == 384
    calls = {"n": 0}

    def crashing(f):
        calls["n"] += 1
        if calls["n"] == 2:
            raise RuntimeError("worker lost")
        return _records(f)

    again = ResumableCampaign(str(tmp_path / "b"), fl, K)   # reopened: continues at 384
    assert again.done == 384
    with pytest.raises(RuntimeError):
        again.run(crashing, 100)
    assert again.done == 484                                  # the chunk that raised is not counted
    last = ResumableCampaign(str(tmp_path / "b"), fl, K)
    assert last.run(_records, 300) == len(fl)
    assert np.array_equal(np.load(str(tmp_path / "b" / "records.npy")), np.load(str(tmp_path / "a" / "records.npy")))
    prog = json.load(open(tmp_path / "b" / "progress.json"))
    assert prog == {"done": len(fl), "n": len(fl), "K": K, "fingerprint": flips_fingerprint(fl), "setup": {}}
    assert not os.path.exists(tmp_path / "b" / "progress.json.tmp")


def test_another_campaign_is_refused(tmp_path):
    fl = _flips()
    ResumableCampaign(str(tmp_path), fl, K).run(_records, 100, max_chunks=1)
    other = fl.copy()
    other["bit"][7] ^= 1
    with pytest.raises(ValueError):
        ResumableCampaign(str(tmp_path), other, K)
    with pytest.raises(ValueError):
        ResumableCampaign(str(tmp_path), fl, K + 1)
    with pytest.raises(ValueError):
        ResumableCampaign(str(tmp_path), fl[:-1], K)


def test_bad_chunk_results_are_rejected_before_counting(tmp_path):
    fl = _flips(100)
    c = ResumableCampaign(str(tmp_path), fl, K)
    with pytest.raises(ValueError):
        c.run(lambda f: _records(f)[:-1], 50)
    with pytest.raises(ValueError):
        c.run(lambda f: np.zeros((len(f), K), dtype=np.float64), 50)
    assert c.done == 0
    with pytest.raises(ValueError):
        c.run(_records, 0)
    with pytest.raises(ValueError):
        ResumableCampaign(str(tmp_path / "x"), np.zeros(4, dtype=np.uint64), K)


def test_another_setup_is_refused(tmp_path):
    """The same upsets against another scene, camera set, guard mode, word mask,
    box or tile shape are another campaign."""
    fl = _flips(200)
    sc = S.make_scene(300, 0, S.FP32, 7)
    cams = S.ring_cameras(K, 64, 48)
    base = dict(planes=sc.planes, fmt=S.FP32, sh_degree=0, cams=cams, guard_mode=-1, word_mask=(1 << 14) - 1)
    setup = campaign_setup(**base)
    ResumableCampaign(str(tmp_path), fl, K, setup).run(_records, 100, max_chunks=1)
    assert ResumableCampaign(str(tmp_path), fl, K, campaign_setup(**base)).done == 100   # same setup: resumes
    other_planes = sc.planes.copy()
    other_planes.view(np.uint32)[3, 5] ^= 1
    lo = np.zeros((14, 300), np.uint32)
    variants = [dict(base, planes=other_planes), dict(base, cams=S.ring_cameras(K, 64, 40)),
                dict(base, guard_mode=0), dict(base, word_mask=1), dict(base, box_lo=lo, box_hi=lo),
                dict(base, tile=(8, 8))]
    for v in variants:
        with pytest.raises(ValueError):
            ResumableCampaign(str(tmp_path), fl, K, campaign_setup(**v))
    with pytest.raises(ValueError):
        ResumableCampaign(str(tmp_path), fl, K)   # no setup given: not this campaign either
