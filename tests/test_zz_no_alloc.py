"""The allocation-free row entry point, for callers that cannot allocate device memory
when they need a result row (their free memory already belongs to another pool, or an
allocation's implicit synchronisation is not acceptable where they run). It must give the
same row as the engine's regular query path, call after call, although every call reuses
the same fixed scratch array inside the library."""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


def _csr(rows, cols, n_rows):
    key = np.unique(rows.astype(np.int64) * (1 << 32) + cols.astype(np.int64))
    r = (key >> 32).astype(np.int64)
    c = (key & 0xFFFFFFFF).astype(np.int32)
    rp = np.zeros(n_rows + 1, np.int64)
    np.cumsum(np.bincount(r, minlength=n_rows), out=rp[1:])
    return rp, c


def test_noalloc_row_matches_engine_twice(cuda_ok):
    import torch
    from paper_2201_04058_b300 import mp
    h = gen.config1_hin()
    s, d = next((s, d) for a, b, s, d in h["relations"] if (a, b) == ("P", "A"))
    n_a, n_p = h["types"]["A"], h["types"]["P"]
    ap_rp, ap_ci = _csr(d, s, n_a)   # authors -> papers
    pa_rp, pa_ci = _csr(s, d, n_p)   # papers -> authors
    # the regular path: APA through mp_submit / mp_result_copy
    eng = mp.Engine(h, policy=mp.MP_POLICY_NONE)
    try:
        rp, ci, val = eng.run({"types": list("APA"), "constraints": []})
    finally:
        eng.close()
    dev = torch.device("cuda", 0)
    y_rp = torch.from_numpy(pa_rp).to(dev)
    y_ci = torch.from_numpy(pa_ci).to(dev)
    cap = n_a
    out_ci = torch.full((cap,), -7, dtype=torch.int32, device=dev)
    out_val = torch.full((cap,), -7, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    degree = np.diff(ap_rp)
    rows = [int(np.argmax(degree)), int(np.nonzero(degree)[0][3])]  # a hub author, then a small one
    for i in rows:
        x = torch.from_numpy(ap_ci[ap_rp[i]:ap_rp[i + 1]].copy()).to(dev)
        rc, nnz = mp.mp_row_product_noalloc(0, stream, x.numel(), x.data_ptr(), 0, y_rp.data_ptr(),
                                            y_ci.data_ptr(), 0, n_a, 0, 0, cap, out_ci.data_ptr(),
                                            out_val.data_ptr())
        assert rc == mp.MP_OK, mp.strerror(rc)
        want_ci = ci[rp[i]:rp[i + 1]]
        want_val = val[rp[i]:rp[i + 1]]
        assert nnz == want_ci.size
        np.testing.assert_array_equal(out_ci[:nnz].cpu().numpy(), want_ci)
        np.testing.assert_array_equal(out_val[:nnz].cpu().numpy().view(np.uint64), want_val)


def test_noalloc_rejects_oversize(cuda_ok):
    import torch
    from paper_2201_04058_b300 import mp
    dev = torch.device("cuda", 0)
    y_rp = torch.tensor([0, 3], dtype=torch.int64, device=dev)
    y_ci = torch.tensor([1, 5, 9], dtype=torch.int32, device=dev)
    x = torch.tensor([0], dtype=torch.int32, device=dev)
    out_ci = torch.zeros(2, dtype=torch.int32, device=dev)
    out_val = torch.zeros(2, dtype=torch.int64, device=dev)
    rc, _ = mp.mp_row_product_noalloc(0, 0, 1, x.data_ptr(), 0, y_rp.data_ptr(), y_ci.data_ptr(), 0,
                                      (1 << 24) + 1, 0, 0, 2, out_ci.data_ptr(), out_val.data_ptr())
    assert rc == mp.MP_ERR_TOO_LARGE
    rc, nnz = mp.mp_row_product_noalloc(0, 0, 1, x.data_ptr(), 0, y_rp.data_ptr(), y_ci.data_ptr(), 0, 10, 0, 0,
                                        2, out_ci.data_ptr(), out_val.data_ptr())
    assert rc == mp.MP_ERR_TOO_LARGE and nnz == 3
    assert out_ci.cpu().tolist() == [0, 0]
    rc, nnz = mp.mp_row_product_noalloc(0, 0, 1, x.data_ptr(), 0, y_rp.data_ptr(), y_ci.data_ptr(), 0, 10, 0, 0,
                                        3, torch.zeros(3, dtype=torch.int32, device=dev).data_ptr(),
                                        torch.zeros(3, dtype=torch.int64, device=dev).data_ptr())
    assert rc == mp.MP_OK and nnz == 3
