"""The library's FP64 evaluations of sin/cos(2 pi u) and ln u for the
53-bit uniforms of its draws (table plus series; the angles in 64-bit fixed
point on the integer units) agree with CUDA's sincospi and log: ln u within
2 ulp; sin and cos within 2 ulp away from their zeros and within 2 ulp of 1
in absolute terms near them; on random words and on the edges of the table
intervals, of the near-one branch and of the range.  Its square root (Newton
steps in fixed point) is within 1 ulp of CUDA's and numpy's, over the whole
range of normal doubles."""
import numpy as np
import pytest

from tests.gpu_common import T, ensure_built, need_gpu, torch

pytestmark = pytest.mark.gpu


def words():
    g = np.random.default_rng(7)
    w = g.integers(0, 2 ** 63, 200000, dtype=np.uint64) * np.uint64(2) + g.integers(0, 2, 200000, dtype=np.uint64)
    k = []
    for i in range(256):                          # table interval edges (k = i 2^45 and neighbours)
        for d in (-1, 0, 1):
            k.append((i << 45) + d)
    top = (1 << 53) - (1 << 46)                    # the near-one branch and its edge
    k += [top - 2, top - 1, top, top + 1, (1 << 53) - 2, (1 << 53) - 1, 0, 1, 2, 3, 1 << 30, 1 << 52]
    k = [x for x in k if 0 <= x < (1 << 53)]
    edge = (np.array(k, dtype=np.uint64) << np.uint64(11)) | np.uint64(0x5A5)
    return np.concatenate([w, edge])


def ulps(a, b):
    scale = np.maximum(np.abs(b), np.finfo(np.float64).tiny)
    return np.abs(a - b) / (np.spacing(scale))


def test_angles_and_logs_match_cuda_within_two_ulp():
    need_gpu()
    ensure_built()
    w = words()
    dw = torch.as_tensor(w.view(np.int64)).cuda()
    out = torch.empty((len(w), 8), dtype=torch.float64, device="cuda")
    T.trmc_fp64_selftest(dw, out)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    # sin and cos: within 2 ulp where they are not small, and within 2 ulp of 1
    # in absolute terms everywhere (the table method cancels near the zeros,
    # where the velocities built from them need absolute, not relative, accuracy)
    for a, b in ((o[:, 0], o[:, 2]), (o[:, 1], o[:, 3])):
        big = np.abs(b) >= 0.05
        assert ulps(a[big], b[big]).max() <= 2.0, ulps(a[big], b[big]).max()
        assert np.abs(a - b).max() <= 2 * np.spacing(1.0), np.abs(a - b).max()
    assert ulps(o[:, 4], o[:, 5]).max() <= 2.0, ulps(o[:, 4], o[:, 5]).max()
    # and against numpy's libm on the same uniforms (independent of both)
    k = (w >> np.uint64(11)).astype(np.float64)
    u = k * 2.0 ** -53
    assert np.abs(o[:, 0] - np.sin(2 * np.pi * u)).max() < 4e-15
    assert np.abs(o[:, 1] - np.cos(2 * np.pi * u)).max() < 4e-15
    uo = (k + 1) * 2.0 ** -53
    assert (np.abs(o[:, 4] - np.log(uo)) <= 4 * np.spacing(np.abs(np.log(uo)) + 1e-300)).all()
    # square root: faithful (within 1 ulp) against CUDA's and numpy's correctly rounded ones
    x = ((w & np.uint64((1 << 52) - 1)) | ((np.uint64(1) + (w >> np.uint64(53)) % np.uint64(2045)) << np.uint64(52))).view(np.float64)
    assert ulps(o[:, 6], o[:, 7]).max() <= 1.0, ulps(o[:, 6], o[:, 7]).max()
    assert ulps(o[:, 6], np.sqrt(x)).max() <= 1.0
    assert np.mean(o[:, 6] == np.sqrt(x)) > 0.99
