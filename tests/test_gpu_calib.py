"""Parity of the drift calibration (step 11) with the oracle on a timeframe
generated with a 1 % faster drift: the vertex time from the FP32 fits agrees
with the FP64 one within 0.01 bins (the per-track FP32 extrapolation moves a
few tracks across the window edges), and both recover the generated scale."""
import pytest

import oracle
import tpcgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_07412_b300 import tpc
    tpc.load()
    return tpc


@pytest.mark.parametrize("eps", [0.0, 0.01])
def test_drift_calibration_parity(lib, eps):
    tf = tpcgen.generate(tpcgen.full_tpc(3, bin_cm=0.5 * (1 + eps)))
    orc = oracle.reconstruct(tf)
    otv, oeps, ot0, on = oracle.calibrate_drift(orc, 250.0)
    with lib.Reconstructor.for_timeframe(tf) as R:
        t = R.submit(tf.pages, tf.page_offsets, tf.n_time_bins)
        R.wait(t)
        tv, e, t0, n = lib.tpc_calibrate_drift(R.ctx, t, 250.0)
        lib.tpc_release(R.ctx, t)
    print(f"eps {eps}: gpu t_v {tv:.5f} eps {e:.6f} n {n}; oracle t_v {otv:.5f} eps {oeps:.6f} n {on}")
    assert abs(n - on) <= 0.01 * on
    assert tv == pytest.approx(otv, abs=0.01)
    assert e == pytest.approx(eps, abs=2e-4) and oeps == pytest.approx(eps, abs=2e-4)
    assert t0 == pytest.approx(tv - 500.0, abs=1e-9)
