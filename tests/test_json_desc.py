"""chem_create_from_json: the library's own reading of the JSON description compiles to the same plan as
the flat-array description (host-only handles, no GPU), and malformed or inconsistent text is rejected
with CHEM_EINVAL."""
import json

import numpy as np
import pytest

from paper_2311_14941_gb300 import chem, synth

MECHS = {"small": synth.mechanism_small, "mid": synth.mechanism_methane_sized, "large": synth.mechanism_large}


@pytest.mark.parametrize("name", list(MECHS))
def test_json_and_struct_descriptions_compile_identically(name):
    m = MECHS[name]()
    a = chem.create(m, device=-1)
    b = chem.create_from_json(m.to_json(), device=-1)
    assert a.info == b.info
    for which in range(11):
        assert np.array_equal(a.export_plan(which), b.export_plan(which)), which
    for x, y in zip(a.jacobian_pattern(), b.jacobian_pattern()):
        assert np.array_equal(x, y)


def test_flat_two_dimensional_fields_and_absent_comp():
    m = synth.mechanism_small()
    d = json.loads(m.to_json())
    for k in ("nasa_lo", "nasa_hi", "troe", "low"):
        d[k] = np.asarray(d[k]).ravel().tolist()
    d["comp"] = None
    b = chem.create_from_json(json.dumps(d), device=-1)
    a = chem.create(m, device=-1)
    assert np.array_equal(a.export_plan(0), b.export_plan(0)) and a.info == b.info


@pytest.mark.parametrize("mutate", [
    lambda d: "{" + json.dumps(d)[1:-1],                       # unterminated object
    lambda d: json.dumps(d)[:-1] + ", }",                      # trailing comma
    lambda d: json.dumps({k: v for k, v in d.items() if k != "A"}),            # missing key
    lambda d: json.dumps(dict(d, b=d["b"][:-1])),                             # inconsistent length
    lambda d: json.dumps(dict(d, reac_sp=[0.5] + d["reac_sp"][1:])),          # non-integer index
    lambda d: json.dumps(dict(d, nasa_lo=d["nasa_lo"][:-1])),                 # short table
    lambda d: json.dumps(d) + " 7",                                           # trailing text
    lambda d: "[1, 2, 3]",                                                    # not an object
])
def test_malformed_json_is_rejected(mutate):
    d = json.loads(synth.mechanism_small().to_json())
    with pytest.raises(chem.ChemError) as ei:
        chem.create_from_json(mutate(d), device=-1)
    assert "status 1" in str(ei.value)


def test_invalid_mechanism_in_valid_json_is_rejected_by_the_compiler():
    d = json.loads(synth.mechanism_small().to_json())
    d["W"][2] = -0.01
    with pytest.raises(chem.ChemError) as ei:
        chem.create_from_json(json.dumps(d), device=-1)
    assert "status 1" in str(ei.value)


def test_mutated_json_never_crashes_and_is_checked():
    """Seeded random edits of a valid description (deleted, inserted or replaced characters, truncation):
    every result is either a compiled handle or CHEM_EINVAL, never a crash or another status."""
    import ctypes
    import random
    L = chem.lib()
    base = synth.mechanism_small().to_json()
    rng = random.Random(2311)
    alphabet = '{}[]",:.-+eE0123456789 \n\tabcdefnulltrue\\/'
    seen = {0: 0, 1: 0}
    for _ in range(600):
        s = list(base)
        for _ in range(rng.randint(1, 6)):
            op, i = rng.random(), rng.randrange(len(s) + 1)
            if op < 0.4 and s:
                del s[min(i, len(s) - 1)]
            elif op < 0.8:
                s.insert(i, rng.choice(alphabet))
            elif s:
                s[min(i, len(s) - 1)] = rng.choice(alphabet)
        if rng.random() < 0.1:
            s = s[:rng.randrange(len(s) + 1)]
        h = ctypes.c_void_p()
        rc = L.chem_create_from_json("".join(s).encode(), -1, ctypes.byref(h))
        assert rc in (0, 1), rc
        seen[rc] += 1
        if rc == 0:
            L.chem_destroy(h)
    assert seen[0] > 0 and seen[1] > 0


@pytest.mark.parametrize("text", [
    '{"W": ' + "[" * 100000 + "]" * 100000 + "}",          # nesting far beyond the reader's limit
    '{"W": ' + '{"a":' * 50000 + "1" + "}" * 50000 + "}",
    '{"W": [1e999]}', '{"W": [1,2,]}', "", "{",
])
def test_pathological_json_is_rejected(text):
    with pytest.raises(chem.ChemError) as ei:
        chem.create_from_json(text, device=-1)
    assert "status 1" in str(ei.value)
