"""Properties of a systematic draw, written from its definition (Sec. III
resampling; offsets as in the library) and independent of both the oracle
and the CUDA path: used where the weights come from the GPU, so the oracle is
never fed GPU output."""
import numpy as np


def check_systematic(idx, w, r: float):
    """idx: the P indices drawn with offset r over weights w (>= 0). Every
    systematic draw has: indices in [0, P) and non-decreasing; every drawn
    particle has positive (quantised) weight; particle p is drawn floor or
    ceil of P q_p / S times (q: weights rounded to multiples of 2^-52, S
    their sum), P draws in all; all-zero weights give the identity."""
    w = np.asarray(w, np.float64)
    idx = np.asarray(idx, np.int64)
    P = len(w)
    assert len(idx) == P
    assert np.all((idx >= 0) & (idx < P))
    assert np.all(np.diff(idx) >= 0)
    q = np.rint(w * 2.0 ** 52) * 2.0 ** -52
    S = q.sum()
    if S == 0:
        assert np.array_equal(idx, np.arange(P))
        return
    assert np.all(q[idx] > 0)
    counts = np.bincount(idx, minlength=P)
    expect = P * q / S
    assert np.all(counts >= np.floor(expect - 1e-9)) and np.all(counts <= np.ceil(expect + 1e-9))
