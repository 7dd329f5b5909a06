"""chem_integrate_noalloc: integration for callers that cannot allocate device memory when they call in.

Such callers are, for example, a CFD code whose memory pool took the device's memory at start-up, or
a time loop that must not pay the implicit device synchronisation of cudaMalloc/cudaFree.  The entry
point keeps its scratch in a fixed array of the library's static device memory.  It runs the same
per-cell code and sorted work queue as chem_integrate in persistent mode, so its results must equal
that entry point's bit for bit -- on a first call and on a second call that finds the previous call's
data still in the shared array.

Collected last on purpose (file name), so a run that stops at the first failure has run everything
else before it; it also passes alone in a fresh process.
"""
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


def _buffers(F, dev, nsub_in):
    N = F.n_cells
    return dict(T=torch.tensor(F.T, device=dev), p=torch.tensor(F.p, device=dev),
                Y=torch.tensor(F.Y.reshape(-1), device=dev), dt=torch.tensor(F.dt, device=dev),
                h_io=torch.zeros(N, dtype=torch.float64, device=dev),
                nsub=torch.tensor(nsub_in, dtype=torch.int32, device=dev),
                status=torch.zeros(N, dtype=torch.int32, device=dev),
                naccept=torch.zeros(N, dtype=torch.int32, device=dev))


def _call(h, F, dev, nsub_in, noalloc, trace_cap=0, **kw):
    b = _buffers(F, dev, nsub_in)
    if trace_cap:
        b["trace"] = torch.zeros(trace_cap * F.n_cells, dtype=torch.float64, device=dev)
    fn = h.integrate_noalloc if noalloc else (lambda *a, **k: h.integrate(*a, mode=1, **k))
    fn(b["T"], b["p"], b["Y"], b["dt"], b["h_io"], b["nsub"], b["status"], naccept=b["naccept"],
       trace=b.get("trace"), **kw)
    torch.cuda.synchronize()
    return {k: b[k].cpu().numpy() for k in ("T", "Y", "h_io", "nsub", "status", "naccept", "trace") if k in b}


_mid = {}


def _mid_handle():
    if not _mid:
        m = synth.mechanism_methane_sized()
        _mid["m"], _mid["h"] = m, chem.create(m, 0)
        _mid["F"] = synth.field_lts_mix(m, 2500, seed=17, dt_range=(1e-7, 1e-4))
    return _mid["m"], _mid["h"], _mid["F"]


@pytest.mark.parametrize("wpc,chunk,method", [(1, 1, 0), (1, 4, 0), (2, 1, 0), (2, 4, 0), (1, 4, 2), (2, 1, 2)])
def test_noalloc_matches_persistent_entry_point_on_two_calls(dev, wpc, chunk, method):
    """One and two warps per cell, one and four cells per queue pull, RODAS3 and RODAS4, with the step trace
    on: the second call of each pair finds the first call's data in the static array."""
    m, h, F = _mid_handle()
    kw = dict(warps_per_cell=wpc, chunk=chunk, method=method, trace_cap=400)
    zeros = np.zeros(F.n_cells, dtype=np.int32)
    ref1 = _call(h, F, dev, zeros, noalloc=False, **kw)
    ref2 = _call(h, F, dev, ref1["nsub"], noalloc=False, **kw)       # second flow step: sorted by the counts
    got1 = _call(h, F, dev, zeros, noalloc=True, **kw)
    got2 = _call(h, F, dev, got1["nsub"], noalloc=True, **kw)        # the static array holds call 1's data
    for ref, got in ((ref1, got1), (ref2, got2)):
        for k in ref:
            assert np.array_equal(ref[k], got[k]), k
    assert len(np.unique(ref1["nsub"])) > 5
    assert np.all(got2["status"] == 0)


def test_noalloc_specialized_matches_persistent_entry_point(dev):
    """The mechanism-specialised kernels behind both entry points: bit-equal results, two calls."""
    m, h, F = _mid_handle()
    h.specialize()
    S = F.subset(np.arange(800))
    kw = dict(warps_per_cell=1, chunk=2, specialized=1)
    zeros = np.zeros(S.n_cells, dtype=np.int32)
    ref1 = _call(h, S, dev, zeros, noalloc=False, **kw)
    got1 = _call(h, S, dev, zeros, noalloc=True, **kw)
    ref2 = _call(h, S, dev, ref1["nsub"], noalloc=False, **kw)
    got2 = _call(h, S, dev, got1["nsub"], noalloc=True, **kw)
    for ref, got in ((ref1, got1), (ref2, got2)):
        for k in ref:
            assert np.array_equal(ref[k], got[k]), k
    assert np.all(got2["status"] == 0)


def test_noalloc_and_persistent_accept_the_largest_chunk(dev):
    """chunk = INT_MAX is reduced to an even share of the cells per lane group: same results as chunk 1."""
    m, h, F = _mid_handle()
    S = F.subset(np.arange(600))
    zeros = np.zeros(S.n_cells, dtype=np.int32)
    base = _call(h, S, dev, zeros, noalloc=False, chunk=1)
    for noalloc in (False, True):
        got = _call(h, S, dev, zeros, noalloc=noalloc, chunk=2**31 - 1)
        for k in base:
            assert np.array_equal(base[k], got[k]), (noalloc, k)


def test_noalloc_takes_no_device_memory_per_call(dev):
    m = synth.mechanism_small()
    h = chem.create(m, 0)
    F = synth.field_uniform_random(m, 512, seed=3)
    zeros = np.zeros(F.n_cells, dtype=np.int32)
    b = _buffers(F, dev, zeros)
    args = (b["T"], b["p"], b["Y"], b["dt"], b["h_io"], b["nsub"], b["status"])
    h.integrate_noalloc(*args)                  # first call on the device: address look-up, module load
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        h.integrate_noalloc(*args)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before


def test_noalloc_rejects_batches_above_its_limit(dev):
    m = synth.mechanism_small()
    h = chem.create(m, 0)
    N = (1 << 20) + 1
    z = lambda n, dt=torch.float64: torch.zeros(n, dtype=dt, device=dev)
    with pytest.raises(chem.ChemError) as ei:
        h.integrate_noalloc(z(N), z(N), z(N * m.n_species), z(N), z(N), z(N, torch.int32), z(N, torch.int32))
    assert "1048576" in str(ei.value) and "status 1" in str(ei.value)
