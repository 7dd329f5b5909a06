"""The Rosenbrock constants of the CUDA source against the oracle's tableaus, on the CPU.

The GPU integrates in the transformed variables U_i = sum_j Gamma_ij k_j (Hairer and Wanner, Sec. IV.7):
a = alpha Gamma^-1, c = diag(1/gamma) - Gamma^-1, m = b Gamma^-1, e = (b - bhat) Gamma^-1.  This test
converts the oracle's k-form tableaus (RODAS3, ROS2, RODAS4) and compares them with the constants typed
into device.cuh, so that a mistyped digit fails here and not only in a GPU parity run.  The bar is
1e-13 relative: the conversion itself rounds at about 1e-15, and a change below 1e-13 in a coefficient
moves no result at the 1e-8 parity tolerance."""
import os
import re

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2311_14941_gb300 import synth

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2311_14941_gb300", "csrc",
                   "device.cuh")


def _constants():
    """name -> value of every `constexpr double NAME = <number or simple expression>` in device.cuh."""
    text = open(SRC).read()
    env = {}
    for decl in re.findall(r"constexpr double ([^;]+);", text):
        for part in re.split(r",\s*(?=[A-Za-z_]\w*\s*=)", decl):
            name, expr = [x.strip() for x in part.split("=", 1)]
            expr = expr.split("//")[0].strip()
            if re.fullmatch(r"0x[0-9a-fA-F.]+p[+-]?\d+", expr):
                env[name] = float.fromhex(expr)
            else:
                env[name] = float(eval(expr, {"__builtins__": {}}, dict(env)))
    return env


def _transformed(t):
    s, g = t["s"], t["gamma"]
    G = t["gam"][:s, :s] + g * np.eye(s)
    Gi = np.linalg.inv(G)
    return dict(a=t["alpha"][:s, :s] @ Gi, c=np.eye(s) / g - Gi, m=t["b"][:s] @ Gi,
                e=(t["b"][:s] - t["bhat"][:s]) @ Gi, gamma=g)


@pytest.fixture(scope="module")
def setup():
    return _constants(), Oracle(synth.mechanism_small())


def _close(x, y):
    return abs(x - y) <= 1e-13 * max(1.0, abs(y))


def test_rodas3_constants(setup):
    k, o = setup
    t = _transformed(o.tableau(0))
    assert _close(k["RG"], t["gamma"])
    a, c, m, e = t["a"], t["c"], t["m"], t["e"]
    for (i, j), name in {(2, 0): "A31", (3, 0): "A41", (3, 2): "A43"}.items():
        assert _close(k[name], a[i, j]), name
    assert max(abs(a[1, 0]), abs(a[2, 1]), abs(a[3, 1])) < 1e-14          # the zeros the kernel exploits
    for (i, j), name in {(1, 0): "C21", (2, 0): "C31", (2, 1): "C32", (3, 0): "C41", (3, 1): "C42",
                         (3, 2): "C43"}.items():
        assert _close(k[name], c[i, j]), name
    assert _close(k["M1"], m[0]) and abs(m[1]) < 1e-14 and _close(k["M3"], m[2]) and _close(k["M4"], m[3])
    assert np.allclose(e, [0, 0, 0, 1], atol=1e-14)


def test_ros2_constants(setup):
    k, o = setup
    t = _transformed(o.tableau(1))
    assert _close(k["RG2"], t["gamma"])
    assert _close(k["R2_A21"], t["a"][1, 0]) and _close(k["R2_C21"], t["c"][1, 0])
    assert _close(k["R2_M1"], t["m"][0]) and _close(k["R2_M2"], t["m"][1])
    assert _close(k["R2_E"], t["e"][0]) and _close(k["R2_E"], t["e"][1])


def test_rodas4_constants(setup):
    k, o = setup
    t = _transformed(o.tableau(2))
    assert _close(k["RG4"], t["gamma"])
    a, c = t["a"], t["c"]
    for i in range(1, 5):
        for j in range(i):
            assert _close(k[f"R4_A{i + 1}{j + 1}"], a[i, j]), (i, j)
    for i in range(1, 6):
        for j in range(i):
            assert _close(k[f"R4_C{i + 1}{j + 1}"], c[i, j]), (i, j)
    # the structure ros4_attempt relies on: stage 6 = stage 5's point + U5, y_new = stage 6's point + U6,
    # error = U6
    assert np.allclose(a[5, :4], a[4, :4], rtol=1e-13) and abs(a[5, 4] - 1.0) < 1e-13
    assert np.allclose(t["m"], [*a[4, :4], 1.0, 1.0], rtol=1e-13, atol=1e-13)
    assert np.allclose(t["e"], [0, 0, 0, 0, 0, 1.0], atol=1e-13)


def _table(name):
    """Entries of `static __constant__ double NAME[r][c] = {{...}, ...};` in device.cuh, as text."""
    text = open(SRC).read()
    body = re.search(name + r"\[(\d+)\]\[(\d+)\]\s*=\s*\{(.*?)\};", text, re.S)
    assert body, name
    rows = re.findall(r"\{([^{}]*)\}", body.group(3))
    return [[x.strip() for x in r.split(",")] for r in rows], int(body.group(1)), int(body.group(2))


def test_rodas4_stage_tables_hold_the_named_coefficients():
    """The stage loop of the RODAS4 attempt reads a_kj and c_kj from two tables: row k - 2 is stage k,
    column j - 1 multiplies U_j, below the diagonal only (a transposed or shifted entry fails here)."""
    for name, letter, nrow in (("kR4A", "A", 4), ("kR4C", "C", 5)):
        rows, r, c = _table(name)
        assert r == nrow and c == nrow and len(rows) == nrow
        for i, row in enumerate(rows):
            assert len(row) == nrow
            for j, x in enumerate(row):
                assert x == (f"R4_{letter}{i + 2}{j + 1}" if j <= i else "0.0"), (name, i, j, x)
