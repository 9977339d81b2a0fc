"""The allocation-free ID entry point against the allocating one.

hssmf_batched_id_noalloc serves callers that must not allocate device
memory while running (allocation synchronizes the device, a memory pool may
own all of it, or a policy forbids it); it keeps its scratch in a fixed
array inside the library.  Collected last so that a failure here comes
after every other test has run; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _inputs(seed, shapes, dt):
    rng = np.random.default_rng(seed)
    Ys = []
    for d_, m_ in shapes:
        r = min(d_, m_)
        Q1, _ = np.linalg.qr(rng.standard_normal((d_, r)))
        Q2, _ = np.linalg.qr(rng.standard_normal((m_, r)))
        Ys.append((Q1 * 10.0 ** (-np.arange(r) / 10.0)) @ Q2.T)
    m = np.array([s[1] for s in shapes], dtype=np.int32)
    d = np.array([s[0] for s in shapes], dtype=np.int32)
    y_off = np.cumsum([0] + [a * b for a, b in shapes])[:-1].astype(np.int64)
    p_off = np.cumsum([0] + list(m))[:-1].astype(np.int64)
    x_off = np.cumsum([0] + [mm * mm // 4 + 1 for mm in m])[:-1].astype(np.int64)
    Yd = torch.tensor(np.concatenate([Y.T.reshape(-1) for Y in Ys]), dtype=dt, device="cuda")
    return Yd, m, d, y_off, p_off, x_off


def _call(fn, prec, Yd, m, d, y_off, p_off, x_off, eps, extra=()):
    dt = Yd.dtype
    piv = torch.full((int(m.sum()),), -1, dtype=torch.int32, device="cuda")
    X = torch.zeros(int(sum(mm * mm // 4 + 1 for mm in m)), dtype=dt, device="cuda")
    ranks = np.zeros(len(m), dtype=np.int32)
    lp = lambda a: a.ctypes.data_as(C.c_void_p)
    fn.restype = C.c_int
    st = fn(prec, len(m), C.c_void_p(Yd.data_ptr()), lp(y_off), lp(m), lp(d), C.c_double(eps), lp(ranks),
            C.c_void_p(piv.data_ptr()), lp(p_off), C.c_void_p(X.data_ptr()), lp(x_off), *extra, None)
    return st, ranks, piv.cpu().numpy(), X.cpu().double().numpy()


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_allocating_entry_point_twice(prec):
    import paper_1502_07405_gb300 as P
    dt = torch.float64 if prec == 0 else torch.float32
    eps = 1e-6 if prec == 0 else 1e-4
    tol = 1e-12 if prec == 0 else 1e-5
    # two calls in a row with different batches: the shared array is reused
    for seed, shapes in ((1, [(192, 128), (256, 300), (64, 64)]), (2, [(128, 128)] * 5 + [(300, 40)])):
        args = _inputs(seed, shapes, dt)
        st0, r0, p0, X0 = _call(P.lib.hssmf_batched_id, prec, *args, eps, extra=(0,))
        st1, r1, p1, X1 = _call(P.lib.hssmf_batched_id_noalloc, prec, *args, eps)
        assert st0 == 0 and st1 == 0
        assert np.array_equal(r0, r1)
        assert np.array_equal(p0, p1)
        assert np.max(np.abs(X1 - X0)) <= tol * max(1.0, np.max(np.abs(X0)))


def test_noalloc_rejects_batches_beyond_its_scratch():
    import paper_1502_07405_gb300 as P
    # 4096 x 2048 doubles = 64 MiB of work copy: above the 32 MiB array
    m = np.array([2048], dtype=np.int32)
    d = np.array([4096], dtype=np.int32)
    z = np.zeros(1, dtype=np.int64)
    Y = torch.zeros(16, dtype=torch.float64, device="cuda")  # never read: rejected first
    piv = torch.zeros(2048, dtype=torch.int32, device="cuda")
    X = torch.zeros(16, dtype=torch.float64, device="cuda")
    ranks = np.zeros(1, dtype=np.int32)
    lp = lambda a: a.ctypes.data_as(C.c_void_p)
    P.lib.hssmf_batched_id_noalloc.restype = C.c_int
    st = P.lib.hssmf_batched_id_noalloc(0, 1, C.c_void_p(Y.data_ptr()), lp(z), lp(m), lp(d), C.c_double(1e-6),
                                        lp(ranks), C.c_void_p(piv.data_ptr()), lp(z),
                                        C.c_void_p(X.data_ptr()), lp(z), None)
    assert st == P.ERR_ARG


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_allocates_no_device_memory(prec):
    """Free device memory is the same before and after each call: the entry
    point uses only its fixed array (the first call on the device, which may
    load the library's device image, is made before measuring)."""
    import paper_1502_07405_gb300 as P
    dt = torch.float64 if prec == 0 else torch.float32
    Yd, m, d, y_off, p_off, x_off = _inputs(3, [(256, 200), (128, 96), (320, 64)], dt)
    piv = torch.full((int(m.sum()),), -1, dtype=torch.int32, device="cuda")
    X = torch.zeros(int(sum(mm * mm // 4 + 1 for mm in m)), dtype=dt, device="cuda")
    ranks = np.zeros(len(m), dtype=np.int32)
    lp = lambda a: a.ctypes.data_as(C.c_void_p)
    fn = P.lib.hssmf_batched_id_noalloc
    fn.restype = C.c_int
    call = lambda: fn(prec, len(m), C.c_void_p(Yd.data_ptr()), lp(y_off), lp(m), lp(d), C.c_double(1e-4),
                      lp(ranks), C.c_void_p(piv.data_ptr()), lp(p_off), C.c_void_p(X.data_ptr()), lp(x_off), None)
    assert call() == 0  # set-up call
    torch.cuda.synchronize()
    for _ in range(3):
        free0 = torch.cuda.mem_get_info()[0]
        assert call() == 0
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
