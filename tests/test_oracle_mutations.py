"""The oracle's pins catch plausible mistakes.

Each case plants one mistake (a flipped sign, a dropped term or factor, a
wrong weight, a swapped operand, the wrong node's wavenumber) in a scratch
copy of ``oracle/`` and runs the pin that should catch it; the pin must
fail.  Opt-in (several minutes): ``HZ_MUTATION_TESTS=1 python -m pytest
tests/test_oracle_mutations.py``.

One change is not listed because it cannot be caught: the coefficient of
the boundary node in the Dirichlet ghost rule (eq. DirchletGhostPoint)
multiplies a value that is zero and not an unknown.
"""

import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.skipif(os.environ.get("HZ_MUTATION_TESTS") != "1",
                                reason="opt-in: HZ_MUTATION_TESTS=1")

OPS = "tests/test_oracle_operators.py::"
SOL = "tests/test_oracle_solver.py::"
KRY = "tests/test_oracle_krylov.py"

# (file under oracle/, original text, planted text, pin that must fail)
MUTATIONS = [
    ("operators.py", "diag = diag - 2j * nsides * np.sqrt(k2) / h",
     "diag = diag + 2j * nsides * np.sqrt(k2) / h",
     OPS + "test_sommerfeld_rows_match_printed_stencils"),
    ("operators.py", "coef = np.where(mirror_out, 2.0 * coef, coef)", "coef = coef",
     OPS + "test_sommerfeld_rows_match_printed_stencils"),
    ("operators.py", "diag = (4.0 * inv_h2 - shift * k2)", "diag = (4.0 * inv_h2 - k2)",
     OPS + "test_cslp_minus_helmholtz_is_imaginary_mass"),
    ("operators.py", "for J, w in ((I - 1, 0.125), (I, 0.75), (I + 1, 0.125)):",
     "for J, w in ((I - 1, 0.25), (I, 0.5), (I + 1, 0.25)):",
     OPS + "test_ho_matches_printed_stencil_and_case_table"),
    ("operators.py", "return (P.T / 4.0).tocsr()", "return (P.T / 2.0).tocsr()",
     OPS + "test_bilinear_and_fw_match_printed"),
    ("operators.py", "        d[:, -1] *= 0.5\n", "        pass\n",
     OPS + "test_DA_symmetric"),
    ("operators.py", "out[key] = out.get(key, 0) + 2j * H * kb * c",
     "out[key] = out.get(key, 0) - 2j * H * kb * c",
     OPS + "test_ghost_rule_reproduces_sommerfeld_rows"),
    ("operators.py",
     "            for d in (ox, oy):\n                for key, c in d.items():\n"
     "                    avg[key] = avg.get(key, 0) + 0.5 * c",
     "            for d in (ox, oy):\n                for key, c in d.items():\n"
     "                    avg[key] = avg.get(key, 0) + c",
     OPS + "test_glk2_dirichlet_laplacian_sine_modes"),
    ("operators.py",
     "            for d in (g[(bi, gj)], g[(gi, bj)]):\n                for key, c in d.items():\n"
     "                    avg[key] = avg.get(key, 0) + 0.5 * c",
     "            for d in (g[(bi, gj)], g[(gi, bj)]):\n                for key, c in d.items():\n"
     "                    avg[key] = avg.get(key, 0) + c",
     OPS + "test_red_cmpo4_sommerfeld_ghost_rule"),
    ("operators.py", "ox = _ghost_rule(bc, H, kb(bi, bj), g[(bi, gj)], g[(ii, gj)])",
     "ox = _ghost_rule(bc, H, kb(bi, gj), g[(bi, gj)], g[(ii, gj)])",
     OPS + "test_glk2_sommerfeld_second_ring_rows_are_consistent"),
    ("operators.py", "    [-98, 56, 980, 56, -98],", "    [-98, 56, 988, 56, -98],",
     OPS + "test_galerkin_ho_matches_printed_glk_stencils"),
    ("operators.py", "    [70, 1960, 4900, 1960, 70],", "    [70, 1960, 4800, 1960, 70],",
     OPS + "test_galerkin_ho_matches_printed_glk_stencils"),
    ("operators.py", "o2_rows = dist <= (0 if variant == 2 else 1)",
     "o2_rows = dist <= (1 if variant == 2 else 1)",
     OPS + "test_glk2_dirichlet_laplacian_sine_modes"),
    ("operators.py", "return lap[dj + 2, di + 2] - mass[dj + 2, di + 2] * k2nb",
     "return lap[dj + 2, di + 2] - mass[dj + 2, di + 2] * coarse.k2[j, i]",
     OPS + "test_red_glk_mass_part_takes_each_nodes_own_wavenumber"),
    ("operators.py", "    return (restriction(Z) @ A0 @ Z).tocsr()",
     "    return (Z.T @ A0 @ Z).tocsr()",
     OPS + "test_galerkin_bilinear_closed_form"),
    ("operators.py", "            return 2.0 * w[R] - k2nb", "            return w[R] - k2nb",
     OPS + "test_red_o6_weights_and_sixth_order"),
    ("solver.py", "self.shift = complex(beta[0], -beta[1])",
     "self.shift = complex(beta[0], beta[1])",
     OPS + "test_cslp_minus_helmholtz_is_imaginary_mass"),
    ("solver.py", "        x = x + self.P[level] @ xc\n", "        x = x - self.P[level] @ xc\n",
     SOL + "test_vcycle_error_propagation_identity"),
    ("solver.py", "        x = x + Dinv * (f - M @ x)\n        return x", "        return x",
     SOL + "test_vcycle_error_propagation_identity"),
    ("solver.py", "self.Dinv = [omega / m.diagonal() for m in self.M]",
     "self.Dinv = [1.0 / m.diagonal() for m in self.M]",
     SOL + "test_vcycle_error_propagation_identity"),
    ("solver.py", "return self.vcycle(v - self.A @ q, 0) + q", "return self.vcycle(v, 0) + q",
     SOL + "test_deflation_invariants"),
    ("solver.py", "return self.Z @ self.coarse_solve(self.RZ @ v)",
     "return self.Z @ self.coarse_solve(2.0 * (self.RZ @ v))",
     SOL + "test_deflation_invariants"),
    ("solver.py", "return w - self.vcycle(self.A @ q, 0) + gamma * q",
     "return w - self.vcycle(self.A @ q, 0)",
     SOL + "test_tlkm_converges_to_the_direct_solution"),
    ("solver.py", "return self.vcycle(v - self.Ed[l] @ q, l) + q", "return self.vcycle(v, l) + q",
     SOL + "test_three_level_deflation_invariant_and_direct_solution"),
    ("solver.py", "q = self.Zd[l] @ self.solve_level(l + 1, self.Rd[l] @ v)",
     "q = self.Zd[l] @ self.solve_level(l + 1, 2.0 * (self.Rd[l] @ v))",
     SOL + "test_multilevel_deflation_invariant_and_direct_solution"),
    ("gradient.py", "return -omega ** 2 - c * 1j * omega", "return -omega ** 2 + c * 1j * omega",
     SOL + "test_gradient_matches_central_differences"),
    ("gradient.py", "x = solve(A, np.conj(g / D))", "x = solve(A, np.conj(g))",
     SOL + "test_gradient_matches_central_differences"),
    ("gradient.py", "grad -= np.real(np.conj(lam) * ap * u)", "grad -= np.real(lam * ap * u)",
     SOL + "test_gradient_matches_central_differences"),
    ("operators.py", "full = (keep @ full_o2 + glk_scale * full_glk).tocsr()",
     "full = (keep @ full_o2 + full_glk).tocsr()",
     SOL + "test_printed_scaling_reproduces_table5_row"),
    ("solver.py", "self.RZ = self.Z.T.tocsr() if printed else ops.restriction(self.Z)",
     "self.RZ = ops.restriction(self.Z)",
     SOL + "test_printed_scaling_reproduces_tables_2_and_3"),
    ("krylov.py", "g[j + 1] = -np.conj(sn[j]) * g[j]", "g[j + 1] = np.conj(sn[j]) * g[j]", KRY),
    ("krylov.py", "H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]",
     "H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]", KRY),
    ("krylov.py", "H[i, j] = np.vdot(V[i], w)", "H[i, j] = np.vdot(w, V[i])", KRY),
    ("krylov.py", "y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]",
     "y[i] = g[i] / H[i, i]", KRY),
    ("krylov.py", "r0 = prec(b - matvec(x0))", "r0 = b - matvec(x0)", KRY),
    ("krylov.py", "            u = u - beta * ui", "            pass", KRY),
    ("krylov.py", "        gamma = np.vdot(c, r)", "        gamma = np.vdot(r, c)", KRY),
    ("krylov.py", "            x = x + prec(sum(y[i] * V[i] for i in range(k)))",
     "            x = x + sum(y[i] * V[i] for i in range(k))", KRY),
    ("krylov.py", "        r0 = b - matvec(x) if np.any(x) else b.copy()",
     "        r0 = b.copy()", KRY),
]


def _scratch(tmp):
    """A copy of the oracle, its CPU tests and the input generators (no
    compiled code) in which the tests import the copied oracle."""
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(tmp, "oracle"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    os.makedirs(os.path.join(tmp, "tests"))
    for f in ("conftest.py", "test_oracle_operators.py", "test_oracle_solver.py",
              "test_oracle_krylov.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(tmp, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(tmp, "tests", "golden"))
    shutil.copytree(os.path.join(ROOT, "paper_2308_06152_gb300"),
                    os.path.join(tmp, "paper_2308_06152_gb300"),
                    ignore=shutil.ignore_patterns("csrc", "*.so", "__pycache__"))


@pytest.mark.parametrize("case", range(len(MUTATIONS)))
def test_pin_catches_planted_mistake(case, tmp_path):
    fname, orig, planted, pin = MUTATIONS[case]
    tmp = str(tmp_path)
    _scratch(tmp)
    path = os.path.join(tmp, "oracle", fname)
    src = open(path).read()
    assert src.count(orig) == 1, f"the text to mutate is not unique in {fname}"
    # the unmutated pin passes ...
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
           "-m", "not gpu", pin]
    if case == 0:
        ok = subprocess.run(cmd, cwd=tmp, capture_output=True, text=True, env=env)
        assert ok.returncode == 0, ok.stdout[-2000:]
    # ... and fails once the mistake is planted
    open(path, "w").write(src.replace(orig, planted))
    bad = subprocess.run(cmd, cwd=tmp, capture_output=True, text=True, env=env)
    assert bad.returncode == 1, (planted, bad.stdout[-2000:])
