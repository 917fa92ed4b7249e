"""Comparison helpers shared by the GPU parity tests."""
import numpy as np

DYN_TOL = 1e-5      # |gpu - oracle| <= DYN_TOL * max(1, |oracle|) per state component
DEPTH_TOL = 1e-4    # |gpu - oracle| <= DEPTH_TOL * oracle on hits


def canon_quat(states: np.ndarray) -> np.ndarray:
    """Flip q -> -q so that w >= 0 (q and -q are the same attitude)."""
    s = np.array(states, dtype=np.float64, copy=True)
    q = s[..., 6:10]
    sign = np.where(q[..., 0:1] < 0, -1.0, 1.0)
    s[..., 6:10] = q * sign
    return s


def dyn_error(gpu: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Scaled error per component: |a - b| / max(1, |b|)."""
    a, b = canon_quat(gpu), canon_quat(ref)
    return np.abs(a - b) / np.maximum(1.0, np.abs(b))


def compare_images(osc, p, states64, depth, rgb, hit, max_tie_frac=0.01):
    """Check GPU images against the oracle.

    Unambiguous pixels: hit id and colour bit-exact, depth within DEPTH_TOL,
    misses exactly max_depth.  Ambiguous pixels (the oracle's stated ties): the
    GPU's answer must be one the ambiguity admits (oracle validator).
    Returns a dict of counts.
    """
    r = osc.render(p, states64)
    tie = r["tie"]
    clear = ~tie
    n_bad_id = int(np.count_nonzero((hit != r["id"]) & clear))
    assert n_bad_id == 0, f"{n_bad_id} unambiguous pixels with a different triangle id"
    assert np.array_equal(rgb[clear], r["rgb"][clear]), "colour differs on unambiguous pixels"
    hitm = clear & (r["id"] >= 0)
    rel = np.abs(depth[hitm].astype(np.float64) - r["depth"][hitm]) / r["depth"][hitm]
    assert rel.size == 0 or rel.max() <= DEPTH_TOL, f"depth rel err {rel.max()}"
    missm = clear & (r["id"] < 0)
    assert np.all(depth[missm] == np.float32(p["max_depth"]))
    assert np.all(rgb[missm] == 0)
    # colour is always the colour of the reported triangle
    tp = np.flatnonzero(tie.reshape(-1))
    if tp.size:
        ok = osc.validate(p, states64, tp, hit.reshape(-1)[tp], depth.reshape(-1)[tp])
        assert ok.all(), f"{int((~ok).sum())} ambiguous pixels with an inadmissible answer"
    frac = float(tie.mean())
    assert frac < max_tie_frac, f"ambiguous fraction {frac}"
    return {"pixels": int(tie.size), "ties": int(tie.sum()), "max_depth_rel_err": float(rel.max()) if rel.size else 0.0,
            "tie_id_diff": int(np.count_nonzero((hit != r["id"]) & tie)), "hit_frac": float((r["id"] >= 0).mean())}


GRAD_RTOL = 1e-3    # per component, against the FP64 oracle's exact gradient
GRAD_FLOOR = 1e-3   # components below GRAD_FLOOR * max|ref| are held to the floor


def grad_error(g: np.ndarray, ref: np.ndarray, floor: float = GRAD_FLOOR) -> tuple:
    """Worst per-component error of one agent's gradient:
    |g_i - ref_i| / max(|ref_i|, floor * max_j |ref_j|).  Returns (worst, index)."""
    g = np.asarray(g, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    scale = np.maximum(np.abs(ref), floor * max(np.abs(ref).max(), 1e-30))
    r = np.abs(g - ref) / scale
    i = int(np.argmax(r))
    return float(r[i]), i
