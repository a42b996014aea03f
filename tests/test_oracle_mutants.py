"""Strength of the oracle's pins: plant one plausible mistake at a time in a
copy of the oracle source (a transposed operand, a wrong sign, a dropped
term, a wrong index) and check that the pin suite fails on every mutant."""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "tomo_oracle.c")

MUTANTS = {
    "chord: transposed cos/sin": ("double t = x * cs + y * sn;", "double t = x * sn + y * cs;"),
    "bin centre: wrong sign of c": ("double pk = ((double)k + 0.5) - c;", "double pk = ((double)k + 0.5) + c;"),
    "plateau: 1/e for 1/a": ("*len = 1.0 / a;", "*len = 1.0 / e;"),
    "ramp: a+e for a*e": ("*len = (h - del) / (a * e);", "*len = (h - del) / (a + e);"),
    "half width: a-e for a+e": ("double h = 0.5 * (a + e);", "double h = 0.5 * (a - e);"),
    "column index transposed": ("col[e] = iy * nx + ix;", "col[e] = ix * ny + iy;"),
    "SIRT: row weights R dropped": ("r[s * rows + i] = R[i] * (b[s * rows + i] - r[s * rows + i]);",
                                   "r[s * rows + i] = (b[s * rows + i] - r[s * rows + i]);"),
    "SIRT: relaxation lambda dropped": ("x[s * cols + j] += lambda * C[j] * g[s * cols + j];",
                                       "x[s * cols + j] += C[j] * g[s * cols + j];"),
    "SIRT: column weights C dropped": ("x[s * cols + j] += lambda * C[j] * g[s * cols + j];",
                                      "x[s * cols + j] += lambda * g[s * cols + j];"),
    "CGLS: beta inverted": ("double beta = gnew / *gamma;", "double beta = *gamma / gnew;"),
    "CGLS: residual update sign": ("for (int64_t i = 0; i < rows; ++i) r[i] -= alpha * q[i];",
                                  "for (int64_t i = 0; i < rows; ++i) r[i] += alpha * q[i];"),
    "TV gradient: neighbour sign": ("g[j + nx] += mu * dy / t;", "g[j + nx] -= mu * dy / t;"),
    "transpose: wrong row index": ("tci[d] = (int32_t)i;", "tci[d] = (int32_t)(rows - 1 - i);"),
    "normaliser: sum for 1/sum": ("out[i] = s != 0.0 ? 1.0 / s : 0.0;", "out[i] = s != 0.0 ? s : 0.0;"),
    "strip: support without the half bin": ("if (!(del < h + 0.5)) return 0;", "if (!(del < h)) return 0;"),
    "strip: window edge sign": ("double dp = del + 0.5, dm = del - 0.5;", "double dp = del + 0.5, dm = 0.5 - del;"),
    "strip: ramp integral": ("return hm * inv_a + (s - hm) * (h - 0.5 * (s + hm)) / ae;",
                             "return hm * inv_a + (s - hm) * (h - 0.5 * (s - hm)) / ae;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    before, after = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(before) == 1, name
    lib = oracle.build_variant(src.replace(before, after), str(tmp_path / "liboracle_mutant.so"))
    env = dict(os.environ, TOMO_ORACLE_LIB=lib, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-x", "-q", "-p", "no:cacheprovider"], env=env, capture_output=True, text=True,
                       cwd=ROOT, timeout=600)
    assert r.returncode != 0, "pins did not catch: " + name


def test_unmutated_variant_passes(tmp_path):
    """Control: the same build-and-run path with the source unchanged passes."""
    lib = oracle.build_variant(open(SRC).read(), str(tmp_path / "liboracle_same.so"))
    env = dict(os.environ, TOMO_ORACLE_LIB=lib, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-q", "-p", "no:cacheprovider"], env=env, capture_output=True, text=True, cwd=ROOT,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:]


# Mistakes planted in the Python half of the oracle (the preconditioned BB-SIRT
# of Sec. 3.1 and its filter): a mutated copy of the package is put first on
# the path, with the unmodified C library.
PY_SRC = os.path.join(ROOT, "oracle", "__init__.py")
FUB_SRC = os.path.join(ROOT, "oracle", "fubini.py")
PY_MUTANTS = {
    "BB: first step not the FBP weight": ("a0 = math.pi / n_theta if first_step is None",
                                          "a0 = 1.0 / n_theta if first_step is None"),
    "BB: step along the gradient": ("x[s] += a * gn[s]", "x[s] -= a * gn[s]"),
    "BB: BB1 ratio inverted": ("a = ss / sy", "a = sy / ss"),
    "BB: sign of y": ("sy = -alpha[s] * float(np.dot(gp[s], gn[s] - gp[s]))",
                      "sy = alpha[s] * float(np.dot(gp[s], gn[s] - gp[s]))"),
    "filter: Hamming window dropped": ("return R * (0.54 + 0.46 * np.cos(2.0 * math.pi * f))", "return R"),
    "filter: odd ramp taps positive": ("h[odd] = -1.0 / (math.pi * n[odd]) ** 2",
                                       "h[odd] = 1.0 / (math.pi * n[odd]) ** 2"),
}


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_pins_catch_planted_python_mistake(name, tmp_path):
    before, after = PY_MUTANTS[name]
    src = open(PY_SRC).read()
    assert src.count(before) == 1, name
    r = _run_python_variant(tmp_path, src.replace(before, after))
    assert r.returncode != 0, "pins did not catch: " + name


def _run_python_variant(tmp_path, source, fubini_source=None, pins=("test_oracle_pins.py", "bb or ramp or ramlak")):
    pkg = tmp_path / "oracle"
    pkg.mkdir()
    (pkg / "__init__.py").write_text(source)
    (pkg / "fubini.py").write_text(fubini_source if fubini_source is not None else open(FUB_SRC).read())
    (pkg / "tomo_oracle.c").write_text(open(SRC).read())
    env = dict(os.environ, TOMO_ORACLE_LIB=oracle.build(), PYTHONPATH=str(tmp_path) + os.pathsep + ROOT)
    cmd = [sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", pins[0]), "-x", "-q", "-p", "no:cacheprovider"]
    if pins[1]:
        cmd += ["-k", pins[1]]
    return subprocess.run(cmd, env=env, capture_output=True, text=True, cwd=str(tmp_path), timeout=600)


def test_unmutated_python_variant_passes(tmp_path):
    """Control: the copied package, unchanged, passes the same pins."""
    r = _run_python_variant(tmp_path, open(PY_SRC).read())
    assert r.returncode == 0, r.stdout[-2000:]


# Mistakes planted in the Fubini-Radon oracle (Sec. 3): the gridding phase,
# the deapodization, the wrap sign, the radial transform and the FBP weight;
# and in its normal operator: the entry formula, the exact adjoint and the
# SIRT that applies it.
FUB_MUTANTS = {
    "fubini: grid phase conjugated": ("return np.exp(2j * math.pi * np.arange(G) * (G / 2.0 - 0.5) / G)",
                                      "return np.exp(-2j * math.pi * np.arange(G) * (G / 2.0 - 0.5) / G)"),
    "fubini: deapodization dropped": ("return 1.0 / kb_hat(fg.pix() / fg.G, fg.kw, fg.beta())",
                                      "return np.ones(fg.n)"),
    "fubini: wrap sign dropped": ("sx = np.where(((kx - kx % G) // G) % 2 != 0, -1.0, 1.0)",
                                  "sx = np.where(((kx - kx % G) // G) % 2 != 0, 1.0, 1.0)"),
    "fubini: radial transform sign": ("E = np.exp(2j * math.pi * np.multiply.outer(fg.omega(), fg.bins())) / fg.n_p",
                                      "E = np.exp(-2j * math.pi * np.multiply.outer(fg.omega(), fg.bins())) / fg.n_p"),
    "fubini: FBP angular weight": ("return (math.pi / fg.n_theta) * _adjoint_polar(fg, Pq, S)",
                                   "return (1.0 / fg.n_theta) * _adjoint_polar(fg, Pq, S)"),
    "fubini SIRT: step along the gradient": ("            x[s_] += a * g[s_]", "            x[s_] -= a * g[s_]"),
    "fubini SIRT: Hamming window dropped": ("return ramp_density(fg) * (0.54 + 0.46 * np.cos(2.0 * math.pi * fg.omega()))",
                                            "return ramp_density(fg)"),
    "normal: Hankel part dropped": ("h += np.cos(phi - math.pi * ps)", "h += 0.0 * np.cos(phi - math.pi * ps)"),
    "normal: unpaired sample at full weight": ("nu[0] = D[0] / 2.0", "nu[0] = D[0]"),
    "direct adjoint: exponent sign": ("ex = np.exp(2j * math.pi * np.multiply.outer(w * math.cos(th[m]), x))",
                                      "ex = np.exp(-2j * math.pi * np.multiply.outer(w * math.cos(th[m]), x))"),
    "direct FBP: angular weight": ("return math.pi / (fg.n_theta * fg.n_p), ramp_density(fg)",
                                   "return 1.0 / (fg.n_theta * fg.n_p), ramp_density(fg)"),
    "normal SIRT: step along the gradient": ("x[s_] = x[s_] + a * g[s_]", "x[s_] = x[s_] - a * g[s_]"),
}


@pytest.mark.parametrize("name", sorted(FUB_MUTANTS))
def test_pins_catch_planted_fubini_mistake(name, tmp_path):
    before, after = FUB_MUTANTS[name]
    src = open(FUB_SRC).read()
    assert src.count(before) == 1, name
    r = _run_python_variant(tmp_path, open(PY_SRC).read(), src.replace(before, after),
                            ("test_oracle_fubini.py", None))
    assert r.returncode != 0, "pins did not catch: " + name


def test_unmutated_fubini_variant_passes(tmp_path):
    r = _run_python_variant(tmp_path, open(PY_SRC).read(), None, ("test_oracle_fubini.py", None))
    assert r.returncode == 0, r.stdout[-2000:]
