"""The hand-written device math helpers against IEEE results and the error
bounds their comments state, over normal, subnormal, huge and special
arguments (called through hsm_eval_helper).

* recip (Newton-Raphson from the FP32 reciprocal) and sqrt_gs (two coupled
  Goldschmidt steps): within 2^-51 relative of the correctly rounded 1/x and
  sqrt x (a few units in the last place).
* sqrt_nr1 (one Newton-Raphson step): within 1.5e-14 relative.
* erf of Abramowitz and Stegun 7.1.28 in FP32: within 3e-7 of erf plus the
  FP32 evaluation term 9e-6 (1 - erf) + 2^-24; GELU built on it likewise.
1/x and sqrt x are correctly rounded in IEEE arithmetic, so numpy's values
on the host are the exact references; erf comes from scipy in FP64."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _args():
    rng = np.random.default_rng(2303)
    e = rng.integers(-1022, 1024, 200_000)
    mant = 1.0 + rng.random(e.size)
    x = np.ldexp(mant, e)
    x = x[np.isfinite(x)]
    sub = np.ldexp(1.0 + rng.random(2000), -1022) * rng.random(2000) * 0.999  # subnormals
    edge = np.array([np.finfo(np.float64).tiny, 2.0 ** -1074, 2.0 ** -1060, np.finfo(np.float64).max,
                     2.0 ** 1023, 2.0 ** -126, 2.0 ** 127, 2.0 ** 128, 2.0 ** -149, 1.0, 2.0, 3.0, 0.5,
                     np.nextafter(1.0, 2.0), np.nextafter(1.0, 0.0)])
    pos = np.concatenate([x, sub[sub > 0], edge])
    return np.concatenate([pos, -pos])


def _eval(fn, x):
    import torch
    from paper_2303_01760_gb300 import hsm

    xt = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    return hsm.eval_helper(fn, xt).cpu().numpy()


def _rel(y, ref):
    big = np.abs(ref) >= np.finfo(np.float64).tiny
    r = np.zeros_like(ref)
    r[big] = np.abs(y[big] - ref[big]) / np.abs(ref[big])
    return r, big


def test_recip_within_a_few_ulp_and_special_values():
    from paper_2303_01760_gb300 import hsm

    x = _args()
    y = _eval(hsm.HSM_HELPER_RECIP, x)
    with np.errstate(divide="ignore", over="ignore"):
        ref = 1.0 / x
    fin = np.isfinite(ref)
    assert np.array_equal(np.isinf(y), np.isinf(ref))
    assert np.array_equal(np.signbit(y), np.signbit(ref))
    r, big = _rel(y[fin], ref[fin])
    assert r.max() <= 2.0 ** -51, r.max()
    # subnormal results: within two subnormal steps
    assert np.abs(y[fin][~big] - ref[fin][~big]).max(initial=0.0) <= 2.0 ** -1073
    sp = np.array([0.0, -0.0, np.inf, -np.inf, np.nan])
    ys = _eval(hsm.HSM_HELPER_RECIP, sp)
    assert ys[0] == np.inf and ys[1] == -np.inf
    assert ys[2] == 0.0 and not np.signbit(ys[2]) and ys[3] == 0.0 and np.signbit(ys[3])
    assert np.isnan(ys[4])
    print(f"recip: max rel err {r.max():.3e} ({r.max() / 2.0 ** -53:.2f} u)")


@pytest.mark.parametrize("which,bound", [("nr1", 1.5e-14), ("gs", 2.0 ** -51)])
def test_sqrt_helpers_within_their_bounds(which, bound):
    from paper_2303_01760_gb300 import hsm

    fn = hsm.HSM_HELPER_SQRT_NR1 if which == "nr1" else hsm.HSM_HELPER_SQRT_GS
    x = _args()
    x = x[x > 0]
    y = _eval(fn, x)
    ref = np.sqrt(x)
    r = np.abs(y - ref) / ref
    assert r.max() <= bound, (which, r.max())
    sp = np.array([0.0, -0.0, np.inf, -np.inf, -1.0, -2.0 ** -1074, np.nan])
    ys = _eval(fn, sp)
    assert ys[0] == 0.0 and not np.signbit(ys[0]) and ys[1] == 0.0 and np.signbit(ys[1])
    assert ys[2] == np.inf
    assert np.all(np.isnan(ys[3:]))
    print(f"sqrt_{which}: max rel err {r.max():.3e} ({r.max() / 2.0 ** -53:.2f} u)")


def test_erf_as_and_gelu_within_their_bounds():
    special = pytest.importorskip("scipy.special")
    from paper_2303_01760_gb300 import hsm

    x = np.concatenate([np.linspace(0.0, 8.0, 400_001), np.geomspace(1e-30, 1e-2, 2000),
                        np.array([1e30, np.float32(3.4e38)])])
    xf = x.astype(np.float32).astype(np.float64)
    e = _eval(hsm.HSM_HELPER_ERF_AS, xf)
    ref = special.erf(xf)
    bound = 3e-7 + 9e-6 * (1.0 - ref) + 2.0 ** -24
    err = np.abs(e - ref)
    assert np.all(err <= bound), float((err - bound).max())

    z = np.concatenate([np.linspace(-10.0, 10.0, 400_001), np.geomspace(1e-20, 1e3, 2000),
                        -np.geomspace(1e-20, 1e3, 2000)])
    zf = z.astype(np.float32).astype(np.float64)
    g = _eval(hsm.HSM_HELPER_GELU, zf)
    gref = 0.5 * zf * (1.0 + special.erf(zf / np.sqrt(2.0)))
    eb = 1.0 - special.erf(np.abs(zf) / np.sqrt(2.0))
    gbound = 0.5 * np.abs(zf) * (3e-7 + 9e-6 * eb + 3 * 2.0 ** -24) + 2.0 ** -22 * np.abs(gref) + 1e-45
    gerr = np.abs(g - gref)
    assert np.all(gerr <= gbound), float((gerr - gbound).max())
    sp = _eval(hsm.HSM_HELPER_GELU, np.array([np.inf, 0.0, -0.0, np.nan]))
    assert sp[0] == np.inf and sp[1] == 0.0 and sp[2] == 0.0 and np.isnan(sp[3])
    print(f"erf_as: max abs err {err.max():.3e}; gelu: max abs err {gerr.max():.3e}")


def test_fp64_probe_reports_a_plausible_rate():
    from paper_2303_01760_gb300 import hsm

    g, ms = hsm.probe_fp64_peak()
    assert ms > 0.0
    # the FP64 FMA rate of a GB300 is about 1.2 TFLOP/s; allow a wide band
    assert 1e2 < g < 1e5, g
