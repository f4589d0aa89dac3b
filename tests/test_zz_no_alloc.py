"""The allocation-free row entry point, for callers that cannot allocate device memory
when they need a result row (their free memory already belongs to another pool, or an
allocation's implicit synchronisation is not acceptable where they run). It must give
the row the CPU oracle gives, call after call, although every call reuses the same fixed
scratch array inside the library; masks, values, hub rows, overflow and malformed ids
included."""
import numpy as np
import pytest

import gen
from oracle import chain as OC
from oracle.hin import OracleHIN

pytestmark = pytest.mark.gpu


def _bitmap(mask_u8):
    """Bit j of word j // 32 set where mask_u8[j] == 1 (the library's mask layout)."""
    b = np.packbits(np.asarray(mask_u8, np.uint8), bitorder="little")
    b = np.concatenate([b, np.zeros((-b.size) % 4, np.uint8)])
    return b.view(np.uint32)


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


class _Row:
    """Calls mp_row_product_noalloc on device copies of numpy inputs."""

    def __init__(self, y_rp, y_ci, y_val, y_cols, cap):
        import torch
        self.y = (_dev(y_rp), _dev(y_ci), None if y_val is None else _dev(y_val.view(np.int64)))
        self.y_cols = y_cols
        self.cap = cap
        self.out_ci = torch.full((max(cap, 1),), -7, dtype=torch.int32, device="cuda:0")
        self.out_val = torch.full((max(cap, 1),), -7, dtype=torch.int64, device="cuda:0")

    def __call__(self, x_ci, x_val=None, km=None, cm=None):
        import torch
        from paper_2201_04058_b300 import mp
        x = _dev(np.asarray(x_ci, np.int32))
        xv = None if x_val is None else _dev(np.asarray(x_val, np.uint64).view(np.int64))
        kmd = None if km is None else _dev(_bitmap(km))
        cmd = None if cm is None else _dev(_bitmap(cm))
        p = lambda t: 0 if t is None else t.data_ptr()
        stream = torch.cuda.current_stream().cuda_stream
        rc, nnz = mp.mp_row_product_noalloc(0, stream, x.numel(), p(x), p(xv), p(self.y[0]), p(self.y[1]),
                                            p(self.y[2]), self.y_cols, p(kmd), p(cmd), self.cap,
                                            p(self.out_ci), p(self.out_val))
        if rc != mp.MP_OK:
            return rc, None, None
        return rc, self.out_ci[:nnz].cpu().numpy(), self.out_val[:nnz].cpu().numpy().view(np.uint64)


def _oracle_row(x_ci, x_val, Y, km, cm):
    x_ci = np.asarray(x_ci, np.int32)
    X = (np.array([0, x_ci.size], np.int64), x_ci, 1, Y[2],
         None if x_val is None else np.asarray(x_val, np.uint64))
    if X[4] is None:
        X = X[:4]
    rp, ci, val = OC.spgemm(X, Y, kmask=km, cmask=cm)
    return ci, val


@pytest.fixture(scope="module")
def valued():
    """APT (authors x topics) and TPA (topics x authors) with their uint64 counts, from the
    oracle on the 2,000-paper HIN: row products of these are rows of APTPA."""
    h = gen.config1_hin()
    o = OracleHIN(h)
    apt = OC.evaluate(o, {"types": list("APT"), "constraints": []})
    tpa = OC.evaluate(o, {"types": list("TPA"), "constraints": []})
    return h, apt, tpa


def test_noalloc_matches_oracle_masks_values_twice(cuda_ok, valued):
    h, apt, tpa = valued
    n_a, n_t = h["types"]["A"], h["types"]["T"]
    Y = (tpa[0], tpa[1], n_t, n_a, tpa[2])
    call = _Row(tpa[0], tpa[1], tpa[2], n_a, n_a)
    g = gen.stream(77, 1)
    deg = np.diff(apt[0])
    hub = int(np.argmax(deg))
    small = int(np.nonzero((deg > 0) & (deg <= 3))[0][0])
    for i in (hub, small, hub):  # the hub twice: the scratch keeps the previous call's bits
        x_ci = apt[1][apt[0][i]:apt[0][i + 1]]
        x_val = apt[2][apt[0][i]:apt[0][i + 1]]
        for km, cm in ((None, None), ((g.random(n_t) < 0.6).astype(np.uint8), None),
                       (None, (g.random(n_a) < 0.3).astype(np.uint8)),
                       ((g.random(n_t) < 0.5).astype(np.uint8), (g.random(n_a) < 0.5).astype(np.uint8))):
            for xv in (x_val, None):
                rc, ci, val = call(x_ci, xv, km, cm)
                assert rc == 0
                want_ci, want_val = _oracle_row(x_ci, xv, Y, km, cm)
                np.testing.assert_array_equal(ci, want_ci)
                np.testing.assert_array_equal(val, want_val)


def test_noalloc_pattern_rows_match_oracle(cuda_ok):
    """0/1 operands (no values): rows of APA, the hub author first."""
    h = gen.config1_hin()
    o = OracleHIN(h)
    ap_rp, ap_ci = o.rel[("A", "P")]
    pa_rp, pa_ci = o.rel[("P", "A")]
    n_a, n_p = h["types"]["A"], h["types"]["P"]
    call = _Row(pa_rp, pa_ci, None, n_a, n_a)
    deg = np.diff(ap_rp)
    for i in (int(np.argmax(deg)), int(np.nonzero(deg)[0][3])):
        x_ci = ap_ci[ap_rp[i]:ap_rp[i + 1]]
        rc, ci, val = call(x_ci)
        assert rc == 0
        want_ci, want_val = _oracle_row(x_ci, None, (pa_rp, pa_ci, n_p, n_a), None, None)
        np.testing.assert_array_equal(ci, want_ci)
        np.testing.assert_array_equal(val, want_val)


def test_noalloc_overflow_reported(cuda_ok):
    """A count above 2^64 - 1 is MP_ERR_OVERFLOW, as the oracle raises for the same row:
    once through one scalar product (2^40 * 2^30), once through a sum (2^63 + 2^63)."""
    from paper_2201_04058_b300 import mp
    y_rp = np.array([0, 2, 3], np.int64)
    y_ci = np.array([1, 4, 4], np.int32)
    cases = [(np.array([1 << 30, 1 << 30, 1 << 30], np.uint64), np.array([0], np.int32),
              np.array([1 << 40], np.uint64)),
             (np.array([1, 1 << 63, 1 << 63], np.uint64), np.array([0, 1], np.int32),
              np.array([1, 1], np.uint64))]
    for y_val, x_ci, x_val in cases:
        Y = (y_rp, y_ci, 2, 6, y_val)
        with pytest.raises(OC.OracleOverflow):
            _oracle_row(x_ci, x_val, Y, None, None)
        rc, _, _ = _Row(y_rp, y_ci, y_val, 6, 8)(x_ci, x_val)
        assert rc == mp.MP_ERR_OVERFLOW
    # the largest count that fits is exact: (2^63 - 1) + 2^63 = 2^64 - 1
    y_val = np.array([1, (1 << 63) - 1, 1 << 63], np.uint64)
    Y = (y_rp, y_ci, 2, 6, y_val)
    rc, ci, val = _Row(y_rp, y_ci, y_val, 6, 8)(np.array([0, 1], np.int32), np.array([1, 1], np.uint64))
    assert rc == 0
    want_ci, want_val = _oracle_row(np.array([0, 1], np.int32), np.array([1, 1], np.uint64), Y, None, None)
    np.testing.assert_array_equal(ci, want_ci)
    np.testing.assert_array_equal(val, want_val)
    assert int(val[-1]) == (1 << 64) - 1


def test_noalloc_rejects_bad_ids_and_oversize(cuda_ok):
    from paper_2201_04058_b300 import mp
    y_rp = np.array([0, 3], np.int64)
    y_ci = np.array([1, 5, 9], np.int32)
    x = np.array([0], np.int32)
    # wider than the scratch array holds: nothing runs
    rc, _, _ = _Row(y_rp, y_ci, None, (1 << 24) + 1, 2)(x)
    assert rc == mp.MP_ERR_TOO_LARGE
    # more entries than the caller's buffers: the size needed comes back, buffers untouched
    import torch
    call = _Row(y_rp, y_ci, None, 10, 2)
    rc, _, _ = call(x)
    assert rc == mp.MP_ERR_TOO_LARGE
    assert call.out_ci.cpu().tolist() == [-7, -7]
    rc, ci, val = _Row(y_rp, y_ci, None, 10, 3)(x)
    assert rc == 0 and ci.tolist() == [1, 5, 9] and val.tolist() == [1, 1, 1]
    # a column id beyond y_cols, or a negative row id, is rejected without being used
    rc, _, _ = _Row(y_rp, y_ci, None, 6, 3)(x)
    assert rc == mp.MP_ERR_ARG
    rc, _, _ = _Row(y_rp, y_ci, None, 10, 3)(np.array([-1], np.int32))
    assert rc == mp.MP_ERR_ARG
    # and the next good call is exact again
    rc, ci, _ = _Row(y_rp, y_ci, None, 10, 3)(x)
    assert rc == 0 and ci.tolist() == [1, 5, 9]
    torch.cuda.synchronize()
