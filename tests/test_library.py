"""Host-side checks of the C ABI that need no GPU: the library builds for sm_103a, loads, and
exports every entry point include/fastmap.h declares; the binding rejects bad arguments
before any device work."""
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2605_18052_gb300 as fm
from paper_2605_18052_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "fastmap.h")).read()
    return sorted(set(re.findall(r"FM_API[^;(]*?\b(fm_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load_library()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["fm_create_problem", "fm_loss_grad", "fm_irls_weights", "fm_step", "fm_get_poses",
              "fm_destroy_problem", "fm_last_error"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (fm_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    # and the binding knows every one of them
    assert sorted(binding.EXPORTED) == _declared()
    for n in _declared():
        getattr(lib, n)


def test_build_flags_target_sm_103a():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_public_python_surface():
    for name in ["Problem", "Mlp", "Translation", "Rotation", "Schedule", "refine", "epipolar_loss", "EpipolarLoss",
                 "default_options", "translation_options"]:
        assert hasattr(fm, name), name
    from paper_2605_18052_gb300 import learned, metrics, translation  # noqa: F401


def test_default_options(lib):
    o = fm.default_options()
    assert (o.storage, o.loss, o.delta, o.beta1, o.beta2, o.use_graph) == (0, 0, 1e-6, 0.9, 0.999, 1)
    o = fm.default_options(storage="fp16", loss="l1")
    assert (o.storage, o.loss) == (fm.FM_STORE_FP16, fm.FM_LOSS_L1)


def test_create_rejects_bad_host_arguments_without_a_gpu(lib):
    # validation of host-side arguments happens before any CUDA call
    R = np.tile(np.eye(3), (2, 1, 1))
    t = np.array([[0.0, 0, 0], [1.0, 0, 0]])
    x = np.zeros((3, 2), np.float32)
    pid = np.zeros(3, np.int32)
    cases = [
        dict(R=R[:1], t=t[:1], cam_i=[0], cam_j=[1]),            # n_cams < 2
        dict(R=R, t=t, cam_i=[0], cam_j=[0]),                    # cam_i == cam_j
        dict(R=R, t=t, cam_i=[0], cam_j=[2]),                    # camera index out of range
        dict(R=R, t=t, cam_i=[0, 1], cam_j=[1, 0], pid=np.zeros(1, np.int32), xx=np.zeros((1, 2), np.float32)),
    ]
    for c in cases:
        with pytest.raises(fm.FastMapError) as ei:
            fm.Problem(c["R"], c["t"], c["cam_i"], c["cam_j"], c.get("pid", pid), c.get("xx", x),
                       c.get("xx", x))
        assert ei.value.status == -1
    with pytest.raises(fm.FastMapError):
        fm.Problem(R, t, [0], [1], pid, x, x, options=fm.default_options(delta=0.0))
    with pytest.raises(fm.FastMapError):
        fm.Problem(R, t, [0], [1], pid, x, x, options=fm.default_options(beta1=1.0))


def test_translation_rejects_bad_host_arguments_without_a_gpu(lib):
    R = np.tile(np.eye(3), (3, 1, 1))
    t = np.array([[1.0, 0, 0], [0.0, 1.0, 0]])
    o = np.zeros((2, 3, 3))
    good = dict(R=R, cam_i=[0, 1], cam_j=[1, 2], t_rel=t, o_init=o)
    cases = [
        dict(good, cam_j=[1, 1], cam_i=[1, 0]),                # cam_i == cam_j
        dict(good, cam_j=[1, 3]),                             # camera index out of range
        dict(good, t_rel=2.0 * t),                            # not unit length
        dict(good, o_init=np.full((2, 3, 3), np.nan)),        # non-finite centres
        dict(good, R=R[:1], cam_i=[0], cam_j=[0], t_rel=t[:1], o_init=o[:, :1]),  # n_cams < 2
    ]
    for c in cases:
        with pytest.raises(fm.FastMapError) as ei:
            fm.Translation(c["R"], c["cam_i"], c["cam_j"], c["t_rel"], c["o_init"])
        assert ei.value.status == -1
    with pytest.raises(fm.FastMapError):
        fm.Translation(R, [0, 1], [1, 2], t, o, fm.translation_options(lr=0.0))


def test_rotation_rejects_bad_host_arguments_without_a_gpu(lib):
    I = np.eye(3)
    Rz = np.array([[0.0, -1, 0], [1, 0, 0], [0, 0, 1]])
    good = dict(cam_i=[0, 1], cam_j=[1, 2], R_rel=np.stack([I, Rz]), n=3)
    cases = [
        dict(good, cam_j=[1, 3]),                                  # index out of range
        dict(good, cam_i=[0, 2], cam_j=[1, 2]),                    # cam_i == cam_j
        dict(good, R_rel=np.stack([I, 2 * Rz])),                   # not orthonormal
        dict(good, R_rel=np.stack([I, -Rz])),                      # det -1
        dict(good, cam_i=[0], cam_j=[1], R_rel=I[None], n=3),      # camera 2 disconnected
    ]
    for c in cases:
        with pytest.raises(fm.FastMapError) as ei:
            fm.Rotation(c["cam_i"], c["cam_j"], c["R_rel"], c["n"])
        assert ei.value.status == -1


def test_header_compiles_as_c_and_links_without_a_gpu(lib, tmp_path):
    # a plain C caller of the boundary: includes the header, links libfastmap.so, and exercises
    # the calls that need no device (defaults, status strings, argument validation)
    src = tmp_path / "caller.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "fastmap.h"
int main(void) {
    fm_options o;
    fm_default_options(&o);
    if (o.storage != FM_STORE_FP32 || o.loss != FM_LOSS_IRLS || o.refine_focal != 0) return 1;
    double R[18] = {1,0,0, 0,1,0, 0,0,1,  1,0,0, 0,1,0, 0,0,1};
    double t[6] = {0,0,0, 1,0,0};
    int ci[1] = {0}, cj[1] = {0};                 /* cam_i == cam_j: rejected before any CUDA call */
    int pid[2] = {0, 0};
    float x[4] = {0, 0, 0, 0};
    fm_problem *p = NULL;
    fm_status st = fm_create_problem(2, R, t, 1, ci, cj, 2, pid, x, x, 0, &o, NULL, &p);
    if (st != FM_EINVAL || p != NULL) return 2;
    if (strlen(fm_last_error()) == 0 || strlen(fm_status_string(FM_EINVAL)) == 0) return 3;
    fm_translation_options to;
    fm_translation_default_options(&to);
    fm_rotation_options ro;
    fm_rotation_default_options(&ro);
    if (!(to.lr > 0) || !(ro.cg_tol > 0) || fm_mlp_num_params() != 1377) return 4;
    printf("ok\n");
    return 0;
}
''')
    so_dir = os.path.dirname(binding.library_path()) if hasattr(binding, "library_path") else \
        os.path.join(ROOT, "paper_2605_18052_gb300")
    exe = tmp_path / "caller"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-L", so_dir, "-lfastmap", "-o", str(exe)], check=True)
    env = dict(os.environ, LD_LIBRARY_PATH=so_dir + ":" + os.environ.get("LD_LIBRARY_PATH", ""))
    out = subprocess.run([str(exe)], capture_output=True, text=True, env=env)
    assert out.returncode == 0 and out.stdout.strip() == "ok", (out.returncode, out.stdout, out.stderr)


def test_missing_library_fails_loudly():
    # a fresh interpreter whose loader points at a path that does not exist: every entry of
    # the product path raises instead of computing anything another way
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import numpy as np\n"
        "import paper_2605_18052_gb300 as fm\n"
        "from paper_2605_18052_gb300 import binding\n"
        "binding.load_library.__defaults__ = ('/nonexistent/libfastmap.so',)\n"
        "R = np.tile(np.eye(3), (2, 1, 1)); t = np.array([[0., 0, 0], [1, 0, 0]])\n"
        "calls = [lambda: fm.Problem(R, t, [0], [1], [0], np.zeros((1, 2), np.float32), np.zeros((1, 2), np.float32)),\n"
        "         lambda: fm.default_options(), lambda: fm.Mlp(np.zeros(1377, np.float32)),\n"
        "         lambda: fm.Rotation([0], [1], np.eye(3)[None], 2)]\n"
        "for f in calls:\n"
        "    try:\n"
        "        f()\n"
        "    except binding.FastMapError as e:\n"
        "        assert 'missing' in str(e), e\n"
        "    else:\n"
        "        raise SystemExit('no error')\n"
        "print('raised')\n" % ROOT)
    r = subprocess.run(["python", "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "raised", r.stdout + r.stderr
