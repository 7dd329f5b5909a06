"""Mechanism-specialised kernels, host side (no GPU): chem_specialize on a host-only handle compiles the
one-warp integration kernels with the run-time compiler into the on-disk cache and loads nothing.

Checked here: the generated source carries the mechanism's sizes (as chem_info reports them) and the
cell layout's extent (chem_info's shared memory per cell) as constants; it compiles for sm_103a (both
kernels, one cubin each in the cache); a second handle of the same mechanism takes the cache (no
compile); a different mechanism gets its own entry; a short buffer is refused with the size needed.
"""
import os
import re

import pytest

from paper_2311_14941_gb300 import chem, synth


def _consts(src):
    return {k: int(v) for k, v in re.findall(r"\b(\w+) = (-?\d+)", src)}


def test_source_holds_the_mechanisms_sizes():
    for mk in (synth.mechanism_small, synth.mechanism_methane_sized, synth.mechanism_large):
        h = chem.create(mk(), device=-1)
        src = h.specialized_source()
        c = _consts(src)
        inf = h.info
        assert c["n"] == inf["n_species"] and c["R"] == inf["n_reactions"] and c["m"] == inf["n_state"]
        assert c["nnz_S"] == inf["nnz_S"] and c["nnz_LU"] == inf["nnz_LU"] and c["n_dslot"] == inf["n_dslots"]
        assert c["lu_steps"] == inf["lu_steps"] and c["sv_steps"] == inf["solve_steps"]
        assert c["n_jpass"] == inf["jac_passes"] and c["width"] == 32
        assert 8 * c["total"] == inf["smem_per_cell"] and c["y"] == 0
        assert '#include "integrate.cuh"' in src


def test_compiles_into_the_cache_and_reuses_it(tmp_path, monkeypatch):
    if not any(os.path.exists(os.path.join(d, "libnvrtc.so.13")) for d in ("/usr/local/cuda/lib64",)):
        pytest.skip("no run-time compiler in this image")
    monkeypatch.setenv("CHEM_RTC_CACHE", str(tmp_path))
    m = synth.mechanism_small()
    h1 = chem.create(m, device=-1)
    t1 = h1.specialize()
    assert t1 > 0.0
    files = sorted(os.listdir(tmp_path))
    assert len(files) == 4 and sum(f.endswith(".cubin") for f in files) == 2
    for f in files:
        assert os.path.getsize(tmp_path / f) > 0
    names = [open(tmp_path / f).read() for f in files if f.endswith(".name")]
    assert any("k_integrate_plain" in n for n in names) and any("k_integrate_persistent" in n for n in names)
    h2 = chem.create(m, device=-1)
    assert h2.specialize() == 0.0          # taken from the cache
    assert sorted(os.listdir(tmp_path)) == files
    # another mechanism's constants differ, so does its key
    h3 = chem.create(synth.mechanism_methane_sized(), device=-1)
    assert h3.specialized_source() != h1.specialized_source()


def test_short_buffer_is_refused_with_the_size():
    import ctypes as C
    h = chem.create(synth.mechanism_small(), device=-1)
    n = C.c_int(16)
    buf = C.create_string_buffer(16)
    rc = chem.lib().chem_specialized_source(h._h, buf, C.byref(n))
    assert rc == 1 and n.value == len(h.specialized_source()) + 1
