"""Persistent work-queue mode (cells sorted by their previous substep count, pulled by resident warps,
launched as one CUDA graph): the same per-cell code as the plain launch, so results must be identical
bit for bit, whatever the order in which cells are taken."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2311_14941_gb300 import chem, synth  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def mid():
    m = synth.mechanism_methane_sized()
    return m, chem.create(m, 0)


def _run(h, F, dev, nsub_in=None, **kw):
    N = F.n_cells
    T = torch.tensor(F.T, device=dev)
    Y = torch.tensor(F.Y.reshape(-1), device=dev)
    hio = torch.zeros(N, dtype=torch.float64, device=dev)
    ns = torch.zeros(N, dtype=torch.int32, device=dev) if nsub_in is None else torch.tensor(nsub_in, device=dev)
    st = torch.zeros(N, dtype=torch.int32, device=dev)
    na = torch.zeros(N, dtype=torch.int32, device=dev)
    h.integrate(T, torch.tensor(F.p, device=dev), Y, torch.tensor(F.dt, device=dev), hio, ns, st, naccept=na, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in dict(T=T, Y=Y, h=hio, nsub=ns, status=st, nacc=na).items()}


def _same(a, b):
    for k in ("T", "Y", "h", "nsub", "status", "nacc"):
        assert np.array_equal(a[k], b[k]), k


def test_persistent_equals_plain_bitwise(mid, dev):
    m, h = mid
    F = synth.field_lts_mix(m, 3000, seed=3, dt_range=(1e-7, 1e-4))
    plain = _run(h, F, dev, mode=0)
    pers = _run(h, F, dev, mode=1)
    _same(plain, pers)
    # second flow step: the previous counts become the sort key
    again = _run(h, F, dev, nsub_in=plain["nsub"], mode=1, chunk=2, block_cells=2)
    _same(plain, again)
    assert len(np.unique(plain["nsub"])) > 5   # a real spread of costs was sorted


def test_persistent_ragged_and_tiny_batches(mid, dev):
    m, h = mid
    F = synth.field_bimodal_jet(m, 16, 16, seed=4)
    for n in (1, 7, 33, 255):
        S = F.subset(np.arange(n))
        _same(_run(h, S, dev, mode=0), _run(h, S, dev, mode=1))


def test_graph_recaptured_when_arguments_change(mid, dev):
    m, h = mid
    F = synth.field_bimodal_jet(m, 8, 8, seed=6)
    a = _run(h, F, dev, mode=1)
    b = _run(h, F, dev, mode=1, rtol=1e-7)          # new options -> new graph
    c = _run(h, F, dev, mode=1)                     # new buffers -> new graph
    _same(a, c)
    assert not np.array_equal(a["nsub"], b["nsub"])


def test_time_budget_reports_timeout(mid, dev):
    """A budget far shorter than the work ends every unfinished cell with TIMEOUT (no hang, no fault);
    the call itself succeeds and the context stays usable."""
    m, h = mid
    F = synth.field_bimodal_jet(m, 32, 32, seed=8)
    for mode in (0, 1):
        r = _run(h, F, dev, mode=mode, time_budget_s=1e-6)
        assert np.all((r["status"] == 5) | (r["status"] == 0))
        assert np.sum(r["status"] == 5) > F.n_cells // 2
        to = r["status"] == 5
        assert np.all(r["nsub"][to] <= 2)
    # the device is still healthy: a normal call afterwards matches the plain result
    _same(_run(h, F, dev, mode=1), _run(h, F, dev, mode=0))


def test_bad_mode_rejected(mid, dev):
    m, h = mid
    F = synth.field_bimodal_jet(m, 4, 4, seed=9)
    with pytest.raises(chem.ChemError):
        _run(h, F, dev, mode=7)


def test_two_warps_per_cell_plain_equals_persistent(mid, dev):
    """With two warps per cell, the plain and the sorted-queue launches give bit-identical results."""
    m, h = mid
    F = synth.field_lts_mix(m, 1500, seed=5, dt_range=(1e-7, 1e-4))
    plain = _run(h, F, dev, mode=0, warps_per_cell=2)
    pers = _run(h, F, dev, mode=1, warps_per_cell=2, block_cells=3)
    _same(plain, pers)
    assert np.all(plain["status"] == 0)
    one = _run(h, F, dev, mode=0, warps_per_cell=1)
    assert np.array_equal(one["status"], plain["status"])


def test_calls_leave_the_callers_current_device(dev):
    """Every entry point runs on its handle's device and puts the caller's current device back."""
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs: a handle on device 1 called while device 0 is current")
    m = synth.mechanism_small()
    h = chem.create(m, 1)
    torch.cuda.set_device(0)
    F = synth.field_uniform_random(m, 8, seed=2)
    d1 = torch.device("cuda", 1)
    T = torch.tensor(F.T, device=d1)
    Y = torch.tensor(F.Y.reshape(-1), device=d1)
    z = lambda dt=torch.float64: torch.zeros(8, dtype=dt, device=d1)
    h.integrate(T, torch.tensor(F.p, device=d1), Y, torch.tensor(F.dt, device=d1), z(), z(torch.int32),
                z(torch.int32), mode=1, stream=torch.cuda.current_stream(d1))
    torch.cuda.synchronize(d1)
    assert torch.cuda.current_device() == 0


@pytest.fixture(scope="module")
def small():
    m = synth.mechanism_small()
    return m, chem.create(m, 0)


def test_two_cells_per_warp_plain_equals_persistent(small, dev):
    """Two cells sharing a warp (16 lanes each): the plain launch and the sorted queue (pairs of
    consecutive queue cells per warp, several chunk sizes and block shapes, ragged cell counts) give
    bit-identical results; they agree with one warp per cell to rounding."""
    m, h = small
    F = synth.field_uniform_random(m, 2049, seed=12)
    F.dt[:] = 10.0 ** np.random.default_rng(3).uniform(-7, -4, F.n_cells)
    plain = _run(h, F, dev, mode=0, cells_per_warp=2)
    for kw in (dict(), dict(chunk=3, block_cells=6), dict(block_cells=3)):
        _same(plain, _run(h, F, dev, mode=1, cells_per_warp=2, **kw))
        _same(plain, _run(h, F, dev, nsub_in=plain["nsub"], mode=1, cells_per_warp=2, **kw))
    for n in (1, 2, 3, 31, 33):
        S = F.subset(np.arange(n))
        _same(_run(h, S, dev, mode=0, cells_per_warp=2), _run(h, S, dev, mode=1, cells_per_warp=2))
    one = _run(h, F, dev, mode=0, warps_per_cell=1, cells_per_warp=1)
    assert np.array_equal(one["status"], plain["status"]) and np.all(plain["status"] == 0)
    same = one["nsub"] == plain["nsub"]
    assert same.mean() > 0.97
    assert np.max(np.abs(one["T"][same] - plain["T"][same]) / one["T"][same]) < 1e-9


def test_two_cells_per_warp_rejects_two_warps(small, dev):
    m, h = small
    F = synth.field_uniform_random(m, 4, seed=1)
    with pytest.raises(chem.ChemError):
        _run(h, F, dev, warps_per_cell=2, cells_per_warp=2)
    with pytest.raises(chem.ChemError):
        _run(h, F, dev, cells_per_warp=3)


def test_automatic_cells_per_warp(small, mid, dev):
    """The automatic choice shares warps for the 10-species mechanism (its half-warp blocks keep more
    cells resident) and not for the 53-species one; the automatic call equals the explicit one."""
    m, h = small
    assert h.info["auto_cells_per_warp"] == 2
    assert h.info["resident_cells"][2] >= h.info["resident_cells"][0]
    assert mid[1].info["auto_cells_per_warp"] == 1
    F = synth.field_uniform_random(m, 300, seed=4)
    _same(_run(h, F, dev, mode=1), _run(h, F, dev, mode=1, cells_per_warp=2))
