"""The oracle's pins are not vacuous: each plausible slip planted in a copy of
the oracle's C source (a sign, a dropped term, a wrong index, a swapped update
order) makes tests/test_oracle.py fail. Runs on the CPU only."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dr_oracle.c")

MUTATIONS = {
    "reaction sign": ("g[3 * b] -= q * d0;", "g[3 * b] += q * d0;"),
    "mass density": ("double me = rhoA * L[e];", "double me = rhoA * L[e] * L[e];"),
    "full-step velocity": ("v[3 * i + r] += 0.5 * dt * a[3 * i + r];\n                u[3 * i + r]",
                           "v[3 * i + r] += dt * a[3 * i + r];\n                u[3 * i + r]"),
    "damping without mass": ("double fd = -c * m[i] * v[3 * i + r];",
                             "double fd = -c * v[3 * i + r];"),
    "engineering strain of length": ("double N = EA[e] * (l / L[e] - 1.0);",
                                     "double N = EA[e] * (l - L[e]);"),
    "stopping rule": ("if (r_norm <= tol * f_ref)", "if (r_norm <= 10.0 * tol * f_ref)"),
    "stress index": ("s[3 * r + c] += q * d[r] * d[c];", "s[3 * r + c] += q * d[r] * d[r];"),
    "stress volume": ("double V = det3(F) * V0;\n    for (int k = 0; k < 9; ++k) sigma[k] = s[k] / V;\n}\n\n/* The same",
                      "double V = V0;\n    for (int k = 0; k < 9; ++k) sigma[k] = s[k] / V;\n}\n\n/* The same"),
    "affine init ignored": ("if (fixed[i] || init == 1) u[3 * i + r] = uaff;",
                            "if (fixed[i]) u[3 * i + r] = uaff;"),
    "kinetic energy without mass": ("ke += 0.5 * m[i] * (v[3 * i] * v[3 * i]",
                                    "ke += 0.5 * (v[3 * i] * v[3 * i]"),
    "internal work without the previous force": ("wi += du * (gp[3 * i + r] + g[3 * i + r]);",
                                                   "wi += du * (2.0 * g[3 * i + r]);"),
    "internal work sign": ("wint -= 0.5 * wi;", "wint += 0.5 * wi;"),
    "damping work half-step": ("double du = dt * v[3 * i + r];", "double du = 0.5 * dt * v[3 * i + r];"),
    "damping work previous force kept": ("fdp[3 * i + r] = fd;", "fdp[3 * i + r] = 0.0;"),
    "residual over all nodes": ("if (fixed[i]) continue;\n            for (int r = 0; r < 3; ++r) {\n                double fd",
                                "for (int r = 0; r < 3; ++r) {\n                double fd"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name!r} not found"
    mutated = src.replace(old, new, 1)
    c_path = tmp_path / "mut.c"
    c_path.write_text(mutated)
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so),
                           str(c_path), "-lm"])
    env = dict(os.environ, FE2_ORACLE_LIB=str(so))
    try:
        res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                              os.path.join(ROOT, "tests", "test_oracle.py")],
                             cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    except subprocess.TimeoutExpired:
        return  # a pin never converges under the mutation: caught
    assert res.returncode != 0, f"mutation {name!r} survived the oracle pins"
