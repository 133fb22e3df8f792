"""The oracle's pins catch planted mistakes.

Each case below plants one plausible mistake (a dropped term, a wrong sign, factor, index or transposed
operand) in a temporary copy of ``oracle/`` and runs the pin file that should catch it against that copy;
the case passes when the pin file fails.  A control run of every pin file against the unmodified copy
must pass, so a failure cannot come from the copy itself.  Nothing here touches the repository's own
``oracle/`` or any GPU.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (oracle file, text, replacement, pin file that must fail, what the mistake is)
CASES = [
    ("transform.py", "return np.tensordot(W, a, axes=(1, 0)) / m", "return np.tensordot(W, a, axes=(1, 0))",
     "test_oracle_transform.py", "forward F(M) without 1/m"),
    ("transform.py", "W = np.conj(w[P]).T", "W = w[P].T", "test_oracle_transform.py",
     "inverse F(M) kernel not conjugated"),
    ("transform.py", "np.exp(-2j * np.pi * j / m)", "np.exp(2j * np.pi * j / m)", "test_oracle_transform.py",
     "sign of the DFT exponent"),
    ("elasticity.py", "np.einsum('...j,...i->...ij', xi, v)) / (2 * mu0)",
     "np.einsum('...j,...i->...ij', xi, v)) / mu0", "test_oracle_elasticity.py", "Gamma0: 1/mu0 for 1/(2 mu0)"),
    ("elasticity.py", "c = (lam0 + mu0) / (mu0 * (lam0 + 2 * mu0))", "c = (lam0 + 2 * mu0) / (mu0 * (lam0 + 2 * mu0))",
     "test_oracle_elasticity.py", "Gamma0: wrong Lame combination"),
    ("elasticity.py", "out = out - c * s[..., None, None]", "out = out + c * s[..., None, None]",
     "test_oracle_elasticity.py", "Gamma0: sign of the xi xi term"),
    ("elasticity.py", "C[3, 3] = C[4, 4] = C[5, 5] = mu", "C[3, 3] = C[4, 4] = C[5, 5] = 2 * mu",
     "test_oracle_elasticity.py", "Voigt shear entry 2 mu"),
    ("elasticity.py", "'...ij,...ij->...', eps, eps).real if not", "'...ii,...ii->...', eps, eps).real if not",
     "test_oracle_residual_pin.py", "Frobenius norm without the shear entries"),
    ("scheme.py", "dC = stiff - C0t ", "dC = C0t - stiff ", "test_oracle_scheme.py", "polarization sign"),
    ("scheme.py", "eps_hat[~nz] = E  ", "eps_hat[~nz] = 0.0", "test_oracle_scheme.py", "mean strain not imposed"),
    ("scheme.py", "eps_hat[nz] = -g", "eps_hat[nz] = g", "test_oracle_scheme.py", "sign of -Gamma0"),
    ("scheme.py", "norm0 = np.sqrt(m) * nE if nE > 0 else 1.0", "norm0 = nE if nE > 0 else 1.0",
     "test_oracle_residual_pin.py", "residual without sqrt(m)"),
    ("scheme.py", "h = h @ np.linalg.inv(np.asarray(L, dtype=np.float64))      # rows",
     "h = h @ np.linalg.inv(np.asarray(L, dtype=np.float64)).T      # rows", "test_oracle_transformed.py",
     "transformed pattern: L^-T transposed"),
    ("scheme.py", "eps_hat[nz] = tau_hat[nz] - 2.0 * el.ddot(C0t, g)",
     "eps_hat[nz] = tau_hat[nz] - 1.0 * el.ddot(C0t, g)", "test_oracle_eyre_milton.py",
     "Eyre-Milton: reflection factor 1 for 2"),
    ("scheme.py", "return float(np.einsum('yij,ijkl,ykl->', a, C0t, c))", "return float(np.einsum('yij,yij->', a, c))",
     "test_oracle_cg.py", "CG: Frobenius instead of the C0 inner product"),
    ("scheme.py", "beta = gamma_new / gamma if gamma != 0 else 0.0", "beta = gamma / gamma_new if gamma_new != 0 else 0.0",
     "test_oracle_cg.py", "CG: beta inverted"),
    ("scheme.py", "E[i, j] = E[j, i] = 0.5", "E[i, j] = E[j, i] = 1.0", "test_oracle_effective.py",
     "unit shear load without the engineering 1/2"),
    ("scheme.py", "return (g2 - rho * rho * np.asarray(eps0, dtype=np.float64)) / (1.0 - rho * rho)",
     "return (g2 - rho * np.asarray(eps0, dtype=np.float64)) / (1.0 - rho)", "test_oracle_filter.py",
     "start filter: rho not squared"),
    ("lattice.py", "                add_row(t, bad, 1)\n                continue\n", "                pass\n",
     "test_oracle_lattice.py", "Smith form: divisibility step skipped"),
    ("lattice.py", "p = (grids * scale) @ Rinv.T", "p = (grids * scale) @ Rinv", "test_oracle_lattice.py",
     "pattern: R^-1 transposed"),
    ("lattice.py", "z = np.floor_divide(2 * u + D, 2 * D)", "z = np.floor_divide(u, D)", "test_oracle_lattice.py",
     "generating set: floor instead of rounding"),
    ("lattice.py", "p[2 * p >= m] -= m", "p[2 * p > m] -= m", "test_oracle_lattice.py",
     "pattern: symmetric cell closed on the wrong side"),
    ("analytic.py", "a = np.linalg.solve(f2 * K1 + f1 * K2, rhs)", "a = np.linalg.solve(f1 * K1 + f2 * K2, rhs)",
     "test_oracle_scheme.py", "laminate: volume fractions swapped"),
    ("analytic.py", "pref = np.sqrt(np.prod(l2)) / 2.0", "pref = np.sqrt(np.prod(l2))", "test_oracle_hashin.py",
     "depolarization: prefactor 1/2 dropped"),
    ("warmstart.py", "return np.roll(x, shift=(-off[0], -off[1], -off[2]), axis=(1, 2, 3))",
     "return np.roll(x, shift=(off[0], off[1], off[2]), axis=(1, 2, 3))", "test_oracle_warmstart.py",
     "convolution: shift direction"),
    ("warmstart.py", "vals = np.array([np.asarray(V)[iu] for V in stiff_voigt]) / mu0",
     "vals = np.array([np.asarray(V)[iu] for V in stiff_voigt])", "test_oracle_warmstart.py",
     "features not divided by mu0"),
    ("classic.py", "eh[~nz] = E", "eh[~nz] = 0.0", "test_oracle_scheme.py",
     "tensor-grid scheme: mean strain not imposed"),
]


def _copy(dst):
    """A working tree with its own oracle/ and tests/, the package itself linked (it holds the seeded
    input generators the pins use)."""
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(dst, "tests"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    os.symlink(os.path.join(ROOT, "paper_1605_05712_gb300"), os.path.join(dst, "paper_1605_05712_gb300"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), dst)


def _run(cwd, files):
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1", OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
    p = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider"]
                       + [os.path.join("tests", f) for f in files],
                       cwd=cwd, env=env, capture_output=True, text=True, timeout=600)
    return p.returncode, p.stdout[-2000:]


def test_every_listed_text_is_in_the_oracle():
    for f, old, new, pin, what in CASES:
        src = open(os.path.join(ROOT, "oracle", f)).read()
        assert src.count(old) >= 1, (f, what)


def test_pins_catch_planted_mistakes(tmp_path):
    pins = sorted({c[3] for c in CASES})

    def one(job):
        kind, k = job
        d = tmp_path / ("%s%d" % (kind, k))
        d.mkdir()
        _copy(str(d))
        if kind == "control":          # every pin file passes on the unmodified copy
            rc, out = _run(str(d), [pins[k]])
            return kind, pins[k], pins[k], rc, out
        f, old, new, pin, what = CASES[k]
        path = d / "oracle" / f
        path.write_text(path.read_text().replace(old, new, 1))
        rc, out = _run(str(d), [pin])
        return kind, what, pin, rc, out

    jobs = [("control", k) for k in range(len(pins))] + [("mutant", k) for k in range(len(CASES))]
    with ThreadPoolExecutor(max(1, min(8, os.cpu_count() or 1))) as ex:
        results = list(ex.map(one, jobs))
    bad_control = [(pin, out) for kind, _, pin, rc, out in results if kind == "control" and rc != 0]
    assert not bad_control, "pins fail on the unmodified copy: %s" % bad_control
    missed = [(what, pin, rc) for kind, what, pin, rc, out in results if kind == "mutant" and rc != 1]
    assert not missed, "planted mistakes not caught (rc 1 = a pin failed): %s" % missed
