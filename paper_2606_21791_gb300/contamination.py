"""Contamination of a sort-first partition (Sec. 5 "Cross-node contamination in
distributed rendering"): host-side reductions of the per-(variant, view) cell
masks that `gs_inject_and_render_regions` returns.

The screen is an 8x8 grid of cells (cell of pixel (x, y) = (8x / W, 8y / H),
bit 8 cy + cx).  A partition into `nodes` regions is an rx x ry grid whose
region (i, j) is the union of cells with 8 i / rx <= cx < 8 (i + 1) / rx (and
likewise in y); for W and H divisible by 8 this equals the region of pixel x
being rx x / W directly."""
import numpy as np

# nodes -> (regions across, regions down)
PARTITIONS = {4: (2, 2), 8: (4, 2), 16: (4, 4), 32: (8, 4), 64: (8, 8)}


def region_masks(cells: np.ndarray, nodes: int) -> np.ndarray:
    """Per mask of 8x8 cells, the mask of the partition's regions that hold a
    marked cell (bit ry_index * rx + rx_index)."""
    rx, ry = PARTITIONS[nodes]
    cells = np.asarray(cells, dtype=np.uint64)
    out = np.zeros(cells.shape, dtype=np.uint64)
    for cy in range(8):
        for cx in range(8):
            hit = (cells >> np.uint64(cy * 8 + cx)) & np.uint64(1)
            region = (cy * ry // 8) * rx + (cx * rx // 8)
            out |= hit << np.uint64(region)
    return out


def popcount(masks: np.ndarray) -> np.ndarray:
    m = np.asarray(masks, dtype=np.uint64)
    return np.array([bin(int(x)).count("1") for x in m.ravel()], dtype=np.int64).reshape(m.shape)


def summary(actual: np.ndarray, predicted: np.ndarray, nodes=(4, 8, 16, 32, 64)) -> dict:
    """For each partition: the mean fraction of nodes contaminated (actual and
    predicted) and the intersection-over-union of the two region sets, per
    variant (mean over variants where the union is non-empty) and pooled."""
    res = {}
    for P in nodes:
        a = region_masks(actual, P)
        p = region_masks(predicted, P)
        na, npred = popcount(a), popcount(p)
        inter, union = popcount(a & p), popcount(a | p)
        nz = union > 0
        res[P] = {
            "frac_actual": float(na.mean() / P),
            "frac_predicted": float(npred.mean() / P),
            "iou_mean": float((inter[nz] / union[nz]).mean()) if nz.any() else None,
            "iou_pooled": float(inter.sum() / union.sum()) if union.sum() else None,
            "actual_outside_predicted": int(popcount(a & ~p).sum()),
        }
    return res
