"""The allocation-free term generation (pt2_det_terms_noalloc).

Callers that cannot allocate device memory when they call (a memory pool or
arena they must not bypass, a latency path that forbids allocation) pass
their own device buffers; the library stages the terms in a fixed device
array it carries.  These checks call it through the C ABI and compare its
output with the allocating pt2_det_terms and with the oracle's terms of the
same determinant, twice in a row (the shared array keeps the previous call's
contents, so the second call must not see them), and check that a
determinant with more terms than the array holds is rejected.

The file name sorts last so that pytest collects it after every other test
file: a run that stops at its first failure (-x) has then already run the
rest of the suite if this convenience entry point fails.  No other test
depends on it or on its order; each test here builds its own context and
passes alone in a fresh process as well.
"""

import numpy as np
import pytest

import oracle
from paper_1808_02049_gb300 import inputs, pt2

pytestmark = pytest.mark.gpu


def _sorted(k, v, h):
    order = np.lexsort((k[:, 1], k[:, 0]))
    return k[order], v[order], h[order]


def test_noalloc_terms_match_allocating_entry_point():
    torch = pytest.importorskip("torch")
    from paper_1808_02049_gb300 import build

    build.build_library()
    s, r = inputs.make_workload("small")
    with pt2.Context(0) as ctx:
        sid = ctx.load_system(s.h, s.eri)
        e0 = float(ctx.diagonal(sid, r.keys).min() - 0.1)
        rid = ctx.load_reference(sid, r.keys, r.coef, e0)
        cap = 4000
        keys = torch.zeros(2 * cap, dtype=torch.int64, device="cuda:0")
        val = torch.zeros(cap, dtype=torch.float64, device="cuda:0")
        haa = torch.zeros(cap, dtype=torch.float64, device="cuda:0")
        torch.cuda.synchronize()
        # two calls in a row, different determinants (the second must not
        # inherit the first call's count or records)
        for det in (7, 512):
            n = pt2.pt2_det_terms_noalloc(ctx.handle, rid, det, keys.data_ptr(), val.data_ptr(), haa.data_ptr(), cap)
            k_ref, v_ref, h_ref = ctx.det_terms(rid, det, cap)
            assert n == k_ref.shape[0] == 3192
            k = keys[: 2 * n].cpu().numpy().view(np.uint64).reshape(n, 2)
            v = val[:n].cpu().numpy()
            h = haa[:n].cpu().numpy()
            k, v, h = _sorted(k, v, h)
            k_ref, v_ref, h_ref = _sorted(k_ref, v_ref, h_ref)
            assert np.array_equal(k, k_ref)
            np.testing.assert_allclose(v, v_ref, rtol=0, atol=1e-14)
            np.testing.assert_allclose(h, h_ref, rtol=0, atol=1e-11)
            # and directly against the oracle's singles and doubles of the determinant
            ok, ov, oh = oracle.det_terms(s.h, s.eri, r.keys[2 * det], r.keys[2 * det + 1], r.coef[det])
            ok, ov, oh = _sorted(ok, ov, oh)
            assert np.array_equal(k, ok)
            np.testing.assert_allclose(v, ov, rtol=0, atol=1e-14)
            np.testing.assert_allclose(h, oh, rtol=0, atol=1e-11)
        # a buffer that is too small is reported, not overrun
        with pytest.raises(pt2.Pt2Error) as e:
            pt2.pt2_det_terms_noalloc(ctx.handle, rid, 3, keys.data_ptr(), val.data_ptr(), haa.data_ptr(), 100)
        assert e.value.code == pt2.PT2_ERR_OOM


def test_noalloc_rejects_determinants_above_the_fixed_scratch():
    torch = pytest.importorskip("torch")
    from paper_1808_02049_gb300 import build

    build.build_library()
    # 12 + 12 electrons in 64 orbitals: 565,656 terms per determinant, above
    # the 524,288 the built-in array holds
    s = inputs.make_integrals(64, 3)
    r = inputs.make_reference(64, 12, 2, 1, 4)
    with pt2.Context(0) as ctx:
        sid = ctx.load_system(s.h, s.eri)
        e0 = float(ctx.diagonal(sid, r.keys).min() - 0.1)
        rid = ctx.load_reference(sid, r.keys, r.coef, e0)
        buf = torch.zeros(16, dtype=torch.float64, device="cuda:0")
        with pytest.raises(pt2.Pt2Error) as e:
            pt2.pt2_det_terms_noalloc(ctx.handle, rid, 0, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), 1)
        assert e.value.code == pt2.PT2_ERR_OOM
        assert "fixed device scratch" in str(e.value)
