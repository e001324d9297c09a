"""The oracle's pins catch plausible mistakes: each case copies the oracle package to a
temporary folder, plants one mistake in the copy (a transposed operand, a flipped sign, a
dropped factor, term or projection, a wrong normaliser, an inverted filter or selection, a
wrong rotation formula) and runs the pin tests against the copy in a fresh interpreter; at
least one pin must fail. A control run of the unchanged copy must pass. The real oracle files
are never touched. CPU only."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

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

# (module file, name, text, planted replacement) for the NumPy parts of the oracle
PY_MUTATIONS = [
    ("__init__.py", "threshold floor ignored", "return max(tau_min, tau0 * factor ** r)", "return tau0 * factor ** r"),
    ("__init__.py", "quadratic-form vector flattened column-major", 'v = np.einsum("pr,pc->prc", b, a).reshape(-1, 9)',
     'v = np.einsum("pr,pc->pcr", b, a).reshape(-1, 9)'),
    ("__init__.py", "offsets kept in FP32", "o1 = (x1 - cen[ci]).astype(np.float16)", "o1 = (x1 - cen[ci])"),
    ("__init__.py", "weight scale not applied", "q = (np.asarray(w, dtype=np.float32) * s).astype(np.float16)",
     "q = (np.asarray(w, dtype=np.float32)).astype(np.float16) * s"),
    ("__init__.py", "gauge rotation transposed", "return _geodesic_deg(Rg, Re @ Q)", "return _geodesic_deg(Rg, Re @ Q.T)"),
    ("translation.py", "baseline direction sign", 'return -np.einsum("nba,nb->na", R[np.asarray(cam_j)], t)',
     'return np.einsum("nba,nb->na", R[np.asarray(cam_j)], t)'),
    ("translation.py", "L2 norm in place of L1", "term = np.abs(r).sum(1)", "term = np.sqrt((r * r).sum(1))"),
    ("translation.py", "subgradient not projected", "g_u = (s - uh * (uh * s).sum(1, keepdims=True)) / nrm[:, None]",
     "g_u = s / nrm[:, None]"),
    ("translation.py", "merge keeps the worst run", "best = np.argmin(", "best = np.argmax("),
    ("translation.py", "normalised by the largest norm", "return c / np.linalg.norm(c, axis=1).mean()",
     "return c / np.linalg.norm(c, axis=1).max()"),
    ("rotation.py", "connection blocks not transposed", "vals += [-w_pair * R_rel[p, a, b], -w_pair * R_rel[p, a, b]]",
     "vals += [-w_pair * R_rel[p, a, b], -w_pair * R_rel[p, b, a]]"),
    ("rotation.py", "second column not orthogonalised", "    y -= x * (x * y).sum(1, keepdims=True)\n", ""),
    ("rotation.py", "third column sign", "z = np.cross(x, y)", "z = np.cross(y, x)"),
    ("rotation.py", "6D second vector not orthogonalised", "u = a2 - b1 * (b1 * a2).sum(1, keepdims=True)\n    b2",
     "u = a2\n    b2"),
    ("rotation.py", "geodesic gradient sign", "dd = -0.5 / np.sqrt(1.0 - cc * cc)", "dd = 0.5 / np.sqrt(1.0 - cc * cc)"),
    ("rotation.py", "relative rotation applied on the wrong side", "X = Rr @ R[ci]", "X = R[ci] @ Rr"),
    ("focal.py", "scales of the two images swapped", "si = s[prob.cam_i][prob.pair_id][:, None]",
     "si = s[prob.cam_j][prob.pair_id][:, None]"),
    ("focal.py", "scale gradient not in log space", "return loss, g_pose, g_s * s", "return loss, g_pose, g_s"),
    ("learned.py", "hidden ReLU dropped", "    h1 = np.maximum(z1, 0.0)\n", "    h1 = z1\n"),
    ("learned.py", "cross-entropy gradient sign", "    dz3 = (p - y) / n\n    g = {\"W3\": h2.T @ dz3[:, None], \"b3\": np.array([dz3.sum()])}\n    dh2",
     "    dz3 = (y - p) / n\n    g = {\"W3\": h2.T @ dz3[:, None], \"b3\": np.array([dz3.sum()])}\n    dh2"),
    ("learned.py", "learned weight floor dropped", "w = p / np.maximum(abs_eps, delta)", "w = p / abs_eps"),
    ("learned.py", "pair-relative feature against the global mean", "f[:, 1] = le - mean_log[pair_id]",
     "f[:, 1] = le - le.mean()"),
    ("focal.py", "scale derivative keeps the homogeneous 1", "u1 = np.concatenate([prob.x1, np.zeros((prob.n_pp, 1))], 1)",
     "u1 = np.concatenate([prob.x1, np.ones((prob.n_pp, 1))], 1)"),
    ("focal_vote.py", "intrinsics applied inverted", "s1 = np.stack([f1, f1, np.ones_like(f1)], axis=1)",
     "s1 = np.stack([1.0 / f1, 1.0 / f1, np.ones_like(f1)], axis=1)"),
    ("focal_vote.py", "ratio of the two smallest singular values", "r = sv[:, 0] / sv[:, 1]", "r = sv[:, 1] / sv[:, 2]"),
    ("focal_vote.py", "temperature sign", "out[c] = np.exp((1.0 - r) / tau).sum()", "out[c] = np.exp((r - 1.0) / tau).sum()"),
    ("focal_vote.py", "known focal length read from the other side", "f1 = np.where(k1 > 0, k1, f)",
     "f1 = np.where(k2 > 0, k2, f)"),
    ("translation.py", "camera loss counts only first images",
     "s = np.bincount(cam_i, weights=term, minlength=n) + np.bincount(cam_j, weights=term, minlength=n)",
     "s = 2 * np.bincount(cam_i, weights=term, minlength=n)"),
]

# pin files run against each mutated file
PINS_FOR = {
    "epipolar.c": ["tests/test_oracle.py", "tests/test_oracle_focal.py"],
    "__init__.py": ["tests/test_oracle.py"],
    "translation.py": ["tests/test_oracle_translation.py"],
    "rotation.py": ["tests/test_oracle_rotation.py"],
    "focal.py": ["tests/test_oracle_focal.py"],
    "learned.py": ["tests/test_oracle_learned.py"],
    "focal_vote.py": ["tests/test_oracle_focal_vote.py"],
}
ALL_PINS = ["tests/test_oracle.py", "tests/test_oracle_focal.py", "tests/test_oracle_translation.py",
            "tests/test_oracle_rotation.py", "tests/test_oracle_learned.py", "tests/test_oracle_focal_vote.py"]


def _run_pins(tmp_path, file: str, source: str, pins) -> subprocess.CompletedProcess:
    """Run `pins` against a copy of the oracle package (in tmp_path) whose `file` holds `source`."""
    dst = tmp_path / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), dst,
                    ignore=shutil.ignore_patterns("__pycache__", "*.so", "*.tmp*"))
    (dst / file).write_text(source)
    code = (
        "import sys\n"
        f"sys.path[:0] = [{str(tmp_path)!r}, {ROOT!r}]\n"
        "import oracle\n"
        f"assert oracle.__file__.startswith({str(tmp_path)!r}), oracle.__file__\n"
        "import pytest\n"
        f"sys.exit(pytest.main(['-q', '-x', '-p', 'no:cacheprovider', '-m', 'not gpu', *{list(pins)!r}]))\n")
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    return subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=900,
                          env=env)


def test_planted_mistakes_fail_a_pin_and_the_unchanged_copy_passes(tmp_path):
    cases = [("epipolar.c",) + m for m in MUTATIONS] + list(PY_MUTATIONS)
    for file, name, text, _ in cases:
        n = open(os.path.join(ROOT, "oracle", file)).read().count(text)
        assert n == 1, f"pattern for {name!r} found {n} times in oracle/{file}"
    # controls: the unchanged copy against every group of pins
    cases = [(file, "control", "", "") for file in PINS_FOR] + cases

    def run(k):
        file, name, text, planted = cases[k]
        source = open(os.path.join(ROOT, "oracle", file)).read()
        if name != "control":
            source = source.replace(text, planted)
        work = tmp_path / f"case{k}"
        work.mkdir()
        r = _run_pins(work, file, source, PINS_FOR[file])
        ok = r.returncode == 0 if name == "control" else (r.returncode == 1 and "FAILED" in r.stdout)
        return f"{file}: {name}", ok, r.stdout[-1500:] + r.stderr[-1500:]

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        results = list(ex.map(run, range(len(cases))))
    wrong = [(name, out) for name, ok, out in results if not ok]
    assert not wrong, wrong
