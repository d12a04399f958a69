"""GPU reflected-series pregrid (rift_ile_pregrid, eq. q-time-pregrid) against
the numpy oracle of the same four steps (oracle/precompute.py q_pregrid):

* random complex128 tables, ragged sizes, r = 1 (identity), 3 and 8: every
  fine sample within 1e-12 of the largest |Q|;
* complex64 in and out: within float rounding;
* a physical table (the small two-detector point, band to 512 Hz, native
  4096 Hz): refined x 8, it matches the 32 768 Hz table of the direct sums of
  eq. QUV to 3e-6 of the largest |Q| over the central half of the window
  (the reflection's own error grows towards the window edges);
* a one-sample table, and refused arguments.
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


@pytest.mark.parametrize("shape,r", [((3, 37, 5), 1), ((3, 37, 5), 3), ((2, 164, 4), 8),
                                     ((1, 1311, 10), 8), ((4, 2, 1), 16)])
def test_pregrid_matches_oracle(R, shape, r):
    rng = np.random.default_rng(sum(shape) + r)
    q = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    got = R.rift_ile_pregrid(torch.as_tensor(q).cuda(), r, q_dtype="complex128").cpu().numpy()
    ref = OP.q_pregrid(q, r)
    assert got.shape == ref.shape == (shape[0], r * (shape[1] - 1) + 1, shape[2])
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    # the fine table passes through the native samples
    assert np.max(np.abs(got[:, ::r, :] - q)) <= 1e-12 * np.max(np.abs(q))


def test_pregrid_complex64(R):
    rng = np.random.default_rng(5)
    q = (rng.standard_normal((4, 165, 10)) + 1j * rng.standard_normal((4, 165, 10))).astype(
        np.complex64)
    got = R.rift_ile_pregrid(torch.as_tensor(q).cuda(), 8, q_dtype="complex64").cpu().numpy()
    ref = OP.q_pregrid(q.astype(np.complex128), 8)
    assert got.dtype == np.complex64
    assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref))


def test_pregrid_physical_table_matches_direct_fine_table(R):
    rng = np.random.default_rng(41)
    dets = W.random_l_detectors(rng, 2)
    truth = W.default_truth(rng, 100.0)
    point, exact, info = W.make_point(
        dets=dets, modes=W.MODES10[:4], f_low=20.0, f_max=512.0, df=0.5, rate=4096.0,
        half_window=0.02, snr=30.0, truth=truth, gmst=0.4, d_ref=100.0, rng=rng, noise=True,
        q_dtype=np.complex128)
    n = point["Q"].shape[1]
    native = OP.q_table_direct(exact["freq"], exact["wgt"], exact["hlm"], exact["dk"],
                               point["q_t0"], point["q_dt"], n)
    fine = R.rift_ile_pregrid(torch.as_tensor(native).cuda(), 8, q_dtype="complex128").cpu().numpy()
    direct = OP.q_table_direct(exact["freq"], exact["wgt"], exact["hlm"], exact["dk"],
                               point["q_t0"], point["q_dt"] / 8, 8 * (n - 1) + 1)
    L = fine.shape[1]
    err = np.max(np.abs(fine - direct), axis=(0, 2)) / np.max(np.abs(direct))
    assert np.max(err[L // 4:3 * L // 4]) < 3e-6
    assert np.max(err) < 2e-3


def test_pregrid_one_sample_and_refusals(R):
    q = torch.tensor([[[1.0 + 2.0j, -0.5j]]], dtype=torch.complex128).cuda()
    got = R.rift_ile_pregrid(q, 8, q_dtype="complex128")
    assert got.shape == (1, 1, 2)
    assert torch.allclose(got, q, rtol=0, atol=1e-15)
    for r in (0, 65):
        with pytest.raises(R.RiftError):
            R.rift_ile_pregrid(q, r)
    big = torch.zeros((65, 2, 64), dtype=torch.complex64).cuda()
    with pytest.raises(R.RiftError):
        R.rift_ile_pregrid(big, 2)
