"""The oracle's pins catch plausible mistakes: each case plants one mistake in a copy of the
oracle's C source (a transposed operand, a flipped sign, a dropped factor or term, a wrong
normaliser, an inverted filter, a wrong rotation formula), builds the copy in a temporary
folder and runs the pin tests against it in a fresh interpreter; at least one pin must fail.
A control run of the unchanged copy must pass. The real oracle files are never touched.
CPU only."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "epipolar.c")

# (name, text in epipolar.c, planted replacement)
MUTATIONS = [
    ("relative rotation transposed", "mat_mul_bt(Rj, Ri, Rn);", "mat_mul_bt(Ri, Rj, Rn);"),
    ("relative translation sign",
     "double d[3] = {ci[0] - cj[0], ci[1] - cj[1], ci[2] - cj[2]};",
     "double d[3] = {cj[0] - ci[0], cj[1] - ci[1], cj[2] - ci[2]};"),
    ("translation not normalised",
     "const double th[3] = {tn[0] / nt, tn[1] / nt, tn[2] / nt};\n        hat(th, K);\n        mat_mul(K, Rn, E + 9 * n);",
     "const double th[3] = {tn[0], tn[1], tn[2]};\n        hat(th, K);\n        mat_mul(K, Rn, E + 9 * n);"),
    ("keypoints swapped in the residual", "s += b[r] * E[3 * r + c] * a[c];", "s += a[r] * E[3 * r + c] * b[c];"),
    ("gradient not projected off the unit translation", "gt[k] = (gth[k] - dp * th[k]) / nt;", "gt[k] = gth[k] / nt;"),
    ("translation term of camera j's rotation gradient dropped", "grad[6 * j + k] += gpj[k] + txg[k];",
     "grad[6 * j + k] += gpj[k];"),
    ("centre gradient sign",
     "grad[6 * i + 3 + k] += tmp[k];\n            grad[6 * j + 3 + k] -= tmp[k];",
     "grad[6 * i + 3 + k] -= tmp[k];\n            grad[6 * j + 3 + k] += tmp[k];"),
    ("camera i rotation gradient sign", "grad[6 * i + k] -= gpi[k];", "grad[6 * i + k] += gpi[k];"),
    ("factor 2 of the squared loss dropped", "d = 2.0 * w[p] * e / Z;", "d = w[p] * e / Z;"),
    ("L1 subgradient sign", "d = (e > 0.0 ? 1.0 : (e < 0.0 ? -1.0 : 0.0)) / Z;",
     "d = (e > 0.0 ? -1.0 : (e < 0.0 ? 1.0 : 0.0)) / Z;"),
    ("weight floor dropped", "w[p] = 1.0 / (a > delta ? a : delta);", "w[p] = 1.0 / a;"),
    ("filter inverted", "if (a <= tau) {", "if (a > tau) {"),
    ("normaliser Z = number of image pairs", "const double Z = (double)n_pp;", "const double Z = (double)n_pairs;"),
    ("Rodrigues coefficient", "b = (1.0 - cos(th)) / th2;", "b = (1.0 - cos(th)) / th;"),
    ("rotation increment on the wrong side", "mat_mul(Ex, R + 9 * k, Rn);", "mat_mul(R + 9 * k, Ex, Rn);"),
    ("Adam bias correction off by one step", "const double bc1 = 1.0 - pow(beta1, (double)step);",
     "const double bc1 = 1.0 - pow(beta1, (double)(step + 1));"),
]

PINS = ["tests/test_oracle.py", "tests/test_oracle_focal.py"]


def _run_pins(tmp_path, source: str) -> subprocess.CompletedProcess:
    src = tmp_path / "epipolar.c"
    src.write_text(source)
    code = (
        "import sys\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import oracle\n"
        f"oracle._SRC = {str(src)!r}\n"
        f"oracle._LIB_PATH = {str(tmp_path / '_liboracle_copy.so')!r}\n"
        "oracle._lib = None\n"
        "import pytest\n"
        f"sys.exit(pytest.main(['-q', '-x', '-p', 'no:cacheprovider', '-m', 'not gpu', *{PINS!r}]))\n")
    return subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600)


def test_unchanged_copy_passes_the_pins(tmp_path):
    r = _run_pins(tmp_path, open(SRC).read())
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]


@pytest.mark.parametrize("name,text,planted", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, text, planted):
    source = open(SRC).read()
    assert source.count(text) == 1, f"pattern for {name!r} not found once in the oracle source"
    r = _run_pins(tmp_path, source.replace(text, planted))
    assert r.returncode == 1 and "FAILED" in r.stdout, (name, r.stdout[-3000:], r.stderr[-2000:])
