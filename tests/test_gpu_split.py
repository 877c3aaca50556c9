"""The collision step evaluates the split counts of Alg. 4.2,
Iround(q R) = floor(x) + [u < x - floor(x)] with x = q R as one FP64 multiply
and u = K 2^-53, in integer arithmetic.  It must equal the FP64 evaluation
(numpy's IEEE multiply, floor and compare) exactly: on random probabilities
of every magnitude, on the edges (q = 0, subnormal, 1, 1 - 2^-53; R = 1 and
2^31 - 1; K = 0 and 2^53 - 1), on products that round to even (odd
significands times small R) and on fractions met exactly by u."""
import numpy as np
import pytest

from tests.gpu_common import T, ensure_built, need_gpu, torch

pytestmark = pytest.mark.gpu


def reference(q, R, K):
    x = q * R.astype(np.float64)
    fl = np.floor(x)
    return (fl + (K.astype(np.float64) * 2.0 ** -53 < x - fl)).astype(np.int64)


def cases():
    g = np.random.default_rng(11)
    n = 400000
    q = np.concatenate([g.random(n // 4), 10.0 ** g.uniform(-320, 0, n // 4), 1.0 - g.random(n // 4) * 1e-6,
                        np.exp(-g.uniform(0, 40, n // 4))])
    q = np.clip(q, 0.0, 1.0)
    R = np.concatenate([g.integers(1, 2 ** 31, n // 2), g.integers(1, 2000, n // 2)]).astype(np.int32)
    K = g.integers(0, 2 ** 53, n, dtype=np.uint64)
    # ties of the product: odd significands times small R
    m = 20000
    qt = ((g.integers(2 ** 51, 2 ** 52, m, dtype=np.uint64) * np.uint64(2) + np.uint64(1))
          .astype(np.float64) * 2.0 ** -53)
    Rt = g.choice(np.array([2, 3, 5, 6, 7, 9, 11, 13, 1023, 4097], np.int32), m)
    Kt = g.integers(0, 2 ** 53, m, dtype=np.uint64)
    # u equal to the fraction (the compare is strict)
    x = qt * Rt
    fr = x - np.floor(x)
    Ke = (fr * 2.0 ** 53).astype(np.uint64)
    exact = Ke.astype(np.float64) * 2.0 ** -53 == fr
    edges_q = np.array([0.0, 5e-324, 2.2250738585072014e-308, 1e-300, 0.5, 1.0 - 2.0 ** -53, 1.0, 0.25, 0.75])
    edges_R = np.array([1, 2, 3, 2 ** 31 - 1, 1000, 2 ** 30], np.int32)
    edges_K = np.array([0, 1, 2 ** 52, 2 ** 53 - 1], np.uint64)
    eq, eR, eK = [a.ravel() for a in np.meshgrid(edges_q, edges_R, edges_K, indexing="ij")]
    q = np.concatenate([q, qt, qt[exact], eq])
    R = np.concatenate([R, Rt, Rt[exact], eR]).astype(np.int32)
    K = np.concatenate([K, Kt, Ke[exact], eK]).astype(np.uint64)
    return q, R, K


def test_integer_iround_equals_fp64_iround():
    need_gpu()
    ensure_built()
    q, R, K = cases()
    out = torch.empty(len(q), dtype=torch.int32, device="cuda")
    T.trmc_split_selftest(torch.as_tensor(q).cuda(), torch.as_tensor(R).cuda(),
                          torch.as_tensor(K.view(np.int64)).cuda(), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.int64)
    ref = reference(q, R, K)
    bad = np.nonzero(got != ref)[0]
    assert bad.size == 0, [(q[i], R[i], K[i], got[i], ref[i]) for i in bad[:5]]
