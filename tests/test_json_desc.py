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
