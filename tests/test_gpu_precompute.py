"""GPU precompute of Q, U, V (eq. QUV, the pregrid of eq. q-time-pregrid)
against the direct sums of the oracle:

* small point: every table sample (complex128) within 1e-12 of the largest
  |Q|, U and V within 1e-13;
* the 3G network (K=4, M=10, 16 385 frequencies, nfft = 131 072, 1 311
  samples): sampled rows against the direct sums, the complex64 table within
  float rounding of the fixture's, U/V against the direct sums;
* a point built from the GPU tables gives the same FP64 lnL and FP32-mixed lnZ
  as one built from the fixture's tables;
* invalid grids are refused.
"""
import numpy as np
import pytest

import oracle.precompute as OP
import workload as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_37393_b300 as R
    return R


def small():
    rng = np.random.default_rng(41)
    dets = W.random_l_detectors(rng, 2)
    truth = W.default_truth(rng, 100.0)
    return W.make_point(dets=dets, modes=W.MODES10[:4], f_low=20.0, f_max=512.0, df=0.5,
                        rate=4096.0, half_window=0.02, snr=30.0, truth=truth, gmst=0.4,
                        d_ref=100.0, rng=rng, noise=True, q_dtype=np.complex128)


def run(R, point, exact, q_dtype):
    df = float(exact["freq"][1] - exact["freq"][0])
    n = np.asarray(point["Q"]).shape[1]
    Q, U, V = R.rift_ile_precompute(exact["hlm"], exact["dk"], exact["wgt"], df, point["q_t0"],
                                    point["q_dt"], n, q_dtype=q_dtype)
    return Q.cpu().numpy(), U.cpu().numpy(), V.cpu().numpy()


def test_small_point_matches_direct_sums(R):
    point, exact, info = small()
    Q, U, V = run(R, point, exact, "complex128")
    Qd = OP.q_table_direct(exact["freq"], exact["wgt"], exact["hlm"], exact["dk"],
                           point["q_t0"], point["q_dt"], Q.shape[1])
    assert np.max(np.abs(Q - Qd)) <= 1e-12 * np.max(np.abs(Qd))
    Ud, Vd = OP.uv_direct(exact["wgt"], exact["hlm"])
    s = np.max(np.abs(Ud))
    assert np.max(np.abs(U - Ud)) <= 1e-13 * s
    assert np.max(np.abs(V - Vd)) <= 1e-13 * s
    # reproducible bit for bit
    Q2, U2, V2 = run(R, point, exact, "complex128")
    assert np.array_equal(Q, Q2) and np.array_equal(U, U2) and np.array_equal(V, V2)


@pytest.fixture(scope="module")
def g3():
    return W.config1(n_draws=1 << 16)


def test_3g_tables(R, g3):
    point, exact, info, draws, logw = g3
    Q, U, V = run(R, point, exact, "complex128")
    rows = np.arange(0, Q.shape[1], 41)
    for k in range(point["K"]):
        Qd = OP.q_direct(exact["freq"], exact["wgt"][k], exact["hlm"], exact["dk"][k],
                         point["q_t0"][k] + point["q_dt"] * rows)
        assert np.max(np.abs(Q[k, rows] - Qd)) <= 1e-12 * np.max(np.abs(Qd)), k
    Ud, Vd = OP.uv_direct(exact["wgt"], exact["hlm"])
    s = np.max(np.abs(Ud))
    assert np.max(np.abs(U - Ud)) <= 1e-13 * s
    assert np.max(np.abs(V - Vd)) <= 1e-13 * s
    Q64, _, _ = run(R, point, exact, "complex64")
    ref = np.asarray(point["Q"])
    assert np.max(np.abs(Q64 - ref)) <= 2 ** -23 * np.max(np.abs(ref))


def test_point_from_gpu_tables(R, g3):
    point, exact, info, draws, logw = g3
    Qg, Ug, Vg = run(R, point, exact, "complex64")
    gpu_point = dict(point)
    gpu_point.update(Q=Qg, U=Ug, V=Vg)
    d = R.Draws(draws, logw)
    a = R.rift_ile_lnL(R.Point(point), d, R.FP64).cpu().numpy()
    b = R.rift_ile_lnL(R.Point(gpu_point), d, R.FP64).cpu().numpy()
    assert np.max(np.abs(a - b) / np.maximum(1.0, np.abs(a))) <= 1e-7
    za = R.rift_ile_lnZ(R.Point(point), d, R.FP32_MIXED)
    zb = R.rift_ile_lnZ(R.Point(gpu_point), d, R.FP32_MIXED)
    assert abs(za[0] - zb[0]) <= 1e-4


def test_invalid_grids(R):
    point, exact, info = small()
    df = float(exact["freq"][1] - exact["freq"][0])
    n = np.asarray(point["Q"]).shape[1]
    with pytest.raises(R.RiftError):   # even grid length
        R.rift_ile_precompute(exact["hlm"][:, 1:], exact["dk"][:, 1:], exact["wgt"][:, 1:], df,
                              point["q_t0"], point["q_dt"], n)
    with pytest.raises(R.RiftError):   # 1/(df dt) not an integer
        R.rift_ile_precompute(exact["hlm"], exact["dk"], exact["wgt"], df, point["q_t0"],
                              point["q_dt"] * 1.1, n)


@pytest.mark.parametrize("p_max", [0, 1, 3])
def test_rotation_bank_matches_oracle(R, p_max):
    """The widened Earth-rotation bank (derivative weights, DFT round trip
    with the sidereal phase) against the oracle's numpy round trip."""
    import workload.composite as WC
    rng = np.random.default_rng(11)
    model = WC.ModeModel(rng, WC.MODES4, 20.0, 1024.0)
    freq = W.freq_grid(1024.0, 0.25)
    h = model(freq)
    got = R.rift_ile_rotation_bank(h, 0.25, 2.0, p_max).cpu().numpy()
    ref = OP.rotation_bank_fft(h, 0.25, 2.0, p_max)
    assert got.shape == ref.shape
    # rows of one derivative order share a scale: compare each row to its own maximum
    scale = np.max(np.abs(ref), axis=1, keepdims=True)
    assert np.max(np.abs(got - ref) / scale) <= 1e-12


@pytest.mark.parametrize("p_max", [0, 3, 6])
def test_arm_bank_matches_oracle(R, p_max):
    """The finite-arm bank (Cauchy-integral W_p on the GPU) against the
    oracle's series construction, on 40 km arms up to 2048 Hz."""
    import workload.composite as WC
    rng = np.random.default_rng(12)
    model = WC.ModeModel(rng, WC.MODES4, 20.0, 2048.0)
    freq = W.freq_grid(2048.0, 0.25)
    h = model(freq)
    T = 4.0e4 / W.C_LIGHT
    got = R.rift_ile_arm_bank(h, 0.25, T, p_max).cpu().numpy()
    ref = OP.arm_bank(h, 0.25, T, p_max)
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
