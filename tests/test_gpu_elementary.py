"""The library's table-driven exponential and logarithm (Tang's reductions, 256 entries each) against
CUDA's exp and log and against the host libm, in units in the last place, on random and boundary
arguments."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _ulps(a, b):
    """Distance in units in the last place between non-negative doubles (exact integer arithmetic)."""
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    return np.abs(a.view(np.int64) - b.view(np.int64))


def _args():
    rng = np.random.default_rng(7)
    parts = [rng.uniform(-745.5, 710.0, 1 << 20),
             rng.uniform(-1.0, 1.0, 1 << 18),
             rng.uniform(-60.0, 40.0, 1 << 18),           # ln k_f, ln Kc, Troe exponents
             rng.uniform(-1e-3, 1e-3, 1 << 16),
             np.ldexp(rng.uniform(-1, 1, 1 << 14), rng.integers(-1074, -20, 1 << 14)),
             (np.arange(-3000, 3000) * np.log(2) / 256) + np.repeat([[-1e-13], [0.0], [1e-13]], 2000, 0).ravel(),
             np.array([0.0, -0.0, 1.0, -1.0, 703.99, -703.99, np.nextafter(704.0, 0), 704.0, -704.0, 709.78,
                       -708.39, -745.13, -746.0, 710.0])]
    return np.concatenate(parts)


def test_library_exp_matches_cuda_exp_within_one_ulp():
    from paper_2311_14941_gb300 import chem
    x = _args()
    xd = torch.tensor(x, device="cuda")
    y0 = torch.empty_like(xd)
    y1 = torch.empty_like(xd)
    chem.eval_elementary(0, xd, y0)
    chem.eval_elementary(1, xd, y1)
    torch.cuda.synchronize()
    ours, cuda = y0.cpu().numpy(), y1.cpu().numpy()
    ref = np.exp(x)
    fin = np.isfinite(ref) & (ref > 0)
    assert np.all(np.isfinite(ours[fin]))
    d_cuda = _ulps(ours[fin], cuda[fin])
    d_libm = _ulps(ours[fin], ref[fin])
    assert d_cuda.max() <= 1, (x[fin][np.argmax(d_cuda)], d_cuda.max())
    assert d_libm.max() <= 1, (x[fin][np.argmax(d_libm)], d_libm.max())
    # a different algorithm rounds differently in the last place, but mostly agrees bit for bit
    assert np.mean(d_cuda == 0) > 0.6 and np.mean(d_libm == 0) > 0.6
    # overflow, underflow and the values at the edges are those of the library exp
    edge = ~fin | (np.abs(x) >= 704)
    assert np.array_equal(ours[edge], cuda[edge])


def test_library_exp_special_values():
    from paper_2311_14941_gb300 import chem
    x = torch.tensor([np.inf, -np.inf, np.nan, 1000.0, -1000.0, 0.0], device="cuda", dtype=torch.float64)
    y = torch.empty_like(x)
    chem.eval_elementary(0, x, y)
    out = y.cpu().numpy()
    assert out[0] == np.inf and out[1] == 0.0 and np.isnan(out[2]) and out[3] == np.inf and out[4] == 0.0
    assert out[5] == 1.0


def _log_args():
    rng = np.random.default_rng(8)
    parts = [np.exp(rng.uniform(-700.0, 700.0, 1 << 20)),
             rng.uniform(200.0, 4000.0, 1 << 18),              # ln T
             1.0 + rng.uniform(-1e-2, 1e-2, 1 << 18),          # near 1: ln F_cent, ln P_r
             1.0 + rng.uniform(-1e-9, 1e-9, 1 << 16),
             np.ldexp(1.0, np.arange(-1022, 1024)),
             np.nextafter(np.ldexp(1.0, np.arange(-1021, 1024)), 0.0),
             np.array([1.0, 0.5, 2.0, np.nextafter(1.0, 0.0), np.nextafter(1.0, 2.0), 1e-300, 1e300,
                       np.finfo(np.float64).max, np.finfo(np.float64).tiny])]
    return np.concatenate(parts)


def test_library_log_matches_cuda_log_within_one_ulp():
    from paper_2311_14941_gb300 import chem
    x = _log_args()
    xd = torch.tensor(x, device="cuda")
    y0 = torch.empty_like(xd)
    y1 = torch.empty_like(xd)
    chem.eval_elementary(2, xd, y0)
    chem.eval_elementary(3, xd, y1)
    torch.cuda.synchronize()
    ours, cuda = y0.cpu().numpy(), y1.cpu().numpy()
    ref = np.log(x)
    # same sign and within one ulp (ulp distance of the magnitudes; ln 1 = 0 exactly)
    assert np.array_equal(np.sign(ours), np.sign(ref)) and ours[x == 1.0].tolist() == [0.0] * int(np.sum(x == 1.0))
    d_cuda = _ulps(np.abs(ours), np.abs(cuda))
    d_libm = _ulps(np.abs(ours), np.abs(ref))
    assert d_cuda.max() <= 1, (x[np.argmax(d_cuda)], d_cuda.max())
    assert d_libm.max() <= 1, (x[np.argmax(d_libm)], d_libm.max())
    assert np.mean(d_libm == 0) > 0.9


def test_library_log_special_values():
    from paper_2311_14941_gb300 import chem
    x = torch.tensor([0.0, -1.0, np.inf, np.nan, 5e-324, 1.0], device="cuda", dtype=torch.float64)
    y = torch.empty_like(x)
    chem.eval_elementary(2, x, y)
    out = y.cpu().numpy()
    assert out[0] == -np.inf and np.isnan(out[1]) and out[2] == np.inf and np.isnan(out[3])
    assert out[4] == np.log(5e-324) and out[5] == 0.0


def test_eval_elementary_rejects_bad_arguments():
    from paper_2311_14941_gb300 import chem
    x = torch.zeros(4, device="cuda", dtype=torch.float64)
    with pytest.raises(chem.ChemError):
        chem.eval_elementary(4, x, x)
