"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol include/mfadvr.h declares, and rejects bad arguments before any
device work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "mfadvr.h")).read()
    return sorted(set(re.findall(r"MFADVR_API\s+[\w\s\*]*?\b(mfadvr_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2204_11762_gb300 import mfadvr
    return mfadvr.load_library()


def test_exports_every_declared_symbol(lib):
    from paper_2204_11762_gb300 import mfadvr
    declared = _declared_symbols()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), f"{name} declared but not exported"
    assert sorted(mfadvr.EXPORTS) == declared


def test_only_abi_symbols_are_exported():
    import subprocess
    from paper_2204_11762_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    ours = sorted({l.split()[-1] for l in out.splitlines() if " T " in l and l.split()[-1].startswith("mfadvr")})
    assert ours == _declared_symbols()


def test_status_strings(lib):
    for st in range(-7, 1):
        assert lib.mfadvr_status_string(st)
    assert lib.mfadvr_status_string(-99) == b"unknown status"


def test_null_arguments_rejected_without_a_device(lib):
    from paper_2204_11762_gb300 import mfadvr
    assert lib.mfadvr_create(None, 0, 0) == mfadvr.EINVAL
    h = ctypes.c_void_p()
    assert lib.mfadvr_create(ctypes.byref(h), -1, 0) == mfadvr.EINVAL
    assert lib.mfadvr_load_model(None, None, None) == mfadvr.EINVAL
    assert lib.mfadvr_eval_points(None, 0, None, 1, None, None, None) == mfadvr.EINVAL
    assert lib.mfadvr_render(None, 0, None, None, None, None, None) == mfadvr.EINVAL
    assert lib.mfadvr_unload_model(None, 0) == mfadvr.EINVAL
    assert lib.mfadvr_destroy(None) == mfadvr.OK
    assert b"NULL" in lib.mfadvr_last_error(None)


def test_header_struct_layout_matches_binding():
    """The ctypes mirrors of the public structs have the C layout, and the
    binding's enum constants the header's values (checked by compiling a probe
    against the header)."""
    import subprocess
    import tempfile
    from paper_2204_11762_gb300 import mfadvr
    src = r'''
#include <stddef.h>
#include <stdio.h>
#include "mfadvr.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(mfadvr_model_desc), offsetof(mfadvr_model_desc, ctrl),
         offsetof(mfadvr_model_desc, storage), sizeof(mfadvr_camera));
  printf("%zu %zu %zu\n", sizeof(mfadvr_render_params), offsetof(mfadvr_render_params, tf_rgba),
         offsetof(mfadvr_render_params, shininess));
  printf("%zu %zu %zu %zu\n", sizeof(mfadvr_render_job), offsetof(mfadvr_render_job, params),
         offsetof(mfadvr_render_job, rgba_dev), sizeof(mfadvr_tuning));
  printf("%zu %zu\n", offsetof(mfadvr_model_desc, weights), offsetof(mfadvr_model_desc, render_form));
  printf("%d %d %d %d %d %d %d\n", MFADVR_FORM_AUTO, MFADVR_FORM_BSPLINE, MFADVR_FORM_POWER, MFADVR_QUERY_VALUE,
         MFADVR_QUERY_GRADIENT, MFADVR_QUERY_BOTH, MFADVR_QUERY_HESSIAN);
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    got = [int(x) for x in out]
    M, Cm, R, J = mfadvr.ModelDesc, mfadvr.Camera, mfadvr.RenderParams, mfadvr.RenderJob
    exp = [ctypes.sizeof(M), M.ctrl.offset, M.storage.offset, ctypes.sizeof(Cm),
           ctypes.sizeof(R), R.tf_rgba.offset, R.shininess.offset,
           ctypes.sizeof(J), J.params.offset, J.rgba_dev.offset, ctypes.sizeof(mfadvr.Tuning),
           M.weights.offset, M.render_form.offset,
           mfadvr.FORM_AUTO, mfadvr.FORM_BSPLINE, mfadvr.FORM_POWER, mfadvr.QUERY_VALUE, mfadvr.QUERY_GRADIENT,
           mfadvr.QUERY_BOTH, mfadvr.QUERY_HESSIAN]
    assert got == exp
