"""The C-ABI library builds, loads and exports every entry point of
include/cpr.h; argument validation rejects bad input before any launch; the
product package does not reach into the oracle.  No GPU needed."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "cpr.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cpr_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1709_01619_gb300 import _native
    return _native.load()


def test_library_exports_every_declared_symbol(lib):
    from paper_1709_01619_gb300 import _native
    declared = _declared()
    assert len(declared) >= 14
    assert set(declared) == set(_native.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name
    assert os.path.dirname(_native.library_path()).startswith(ROOT)


def test_struct_layouts_match_the_header(tmp_path):
    """ctypes mirrors of cpr_config / cpr_norms_out against the C compiler's
    layout of include/cpr.h."""
    import shutil
    import subprocess
    from paper_1709_01619_gb300 import _native
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    fields_c = [f for f, _ in _native._Config._fields_]
    fields_n = [f for f, _ in _native._Norms._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cpr.h"', "int main(void){",
             'printf("%zu\\n", sizeof(cpr_config));', 'printf("%zu\\n", sizeof(cpr_norms_out));']
    lines += [f'printf("%zu\\n", offsetof(cpr_config, {f}));' for f in fields_c]
    lines += [f'printf("%zu\\n", offsetof(cpr_norms_out, {f}));' for f in fields_n]
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(_native._Config)
    assert vals[1] == ctypes.sizeof(_native._Norms)
    assert vals[2:2 + len(fields_c)] == [getattr(_native._Config, f).offset for f in fields_c]
    assert vals[2 + len(fields_c):] == [getattr(_native._Norms, f).offset for f in fields_n]


BAD = [
    dict(eqn=7), dict(nx=0), dict(ny=-3), dict(x1=0.0), dict(p=0), dict(p=5), dict(pts=2),
    dict(corr=3), dict(corr=-1), dict(flux=9), dict(div=3), dict(bc_x=4), dict(gamma=1.0), dict(limiter=2),
    dict(tvb_M=-1.0), dict(lim_eps=-1.0), dict(dtype=5), dict(cfl=-0.1),
    dict(eqn=1, flux=1),  # upwind is for linear advection only
    dict(scheme=3),
    dict(scheme=1, p=1),  # FV stores one average per element: p = 0
    dict(scheme=2, p=2),
    dict(scheme=2, p=0, limiter=1),
    dict(scheme=1, p=0, limiter=1),  # FV limits its slopes itself
]


@pytest.mark.parametrize("kw", BAD)
def test_init_rejects_bad_config_before_any_launch(lib, kw):
    from paper_1709_01619_gb300 import _native
    cfg = _native.Config(**kw)
    h = ctypes.c_void_p()
    st = lib.cpr_init(ctypes.byref(cfg._c()), None, ctypes.byref(h))
    assert st == _native.CPR_EINVAL
    assert not h.value
    assert lib.cpr_last_error(None)


def test_null_arguments(lib):
    from paper_1709_01619_gb300 import _native
    assert lib.cpr_init(None, None, None) == _native.CPR_EINVAL
    assert lib.cpr_residual(None, None, None) == _native.CPR_EINVAL
    assert lib.cpr_step(None, None, 1, 0.0, 0.0) == _native.CPR_EINVAL
    assert lib.cpr_norms(None, None, None, None) == _native.CPR_EINVAL
    assert lib.cpr_step_vjp(None, None, None, None, 0.1) == _native.CPR_EINVAL
    assert lib.cpr_step_stages(None, None, None, None, None, 0.1) == _native.CPR_EINVAL
    assert lib.cpr_step_vjp_stages(None, None, None, None, None, None, 0.1) == _native.CPR_EINVAL
    assert lib.cpr_state_elems(None) == 0
    lib.cpr_destroy(None)


def test_roe_flux_passes_validation(lib):
    """Roe's flux is built: init gets past the configuration checks (it then
    needs a device)."""
    from paper_1709_01619_gb300 import _native
    cfg = _native.Config(flux=_native.ROE)
    h = ctypes.c_void_p()
    st = lib.cpr_init(ctypes.byref(cfg._c()), None, ctypes.byref(h))
    assert st in (_native.CPR_OK, _native.CPR_ECUDA)
    if st == _native.CPR_OK:
        lib.cpr_destroy(h)


@pytest.mark.parametrize("kw", [dict(corr=1), dict(corr=2, pts=1), dict(scheme=2, p=0),
                                dict(scheme=1, p=0, corr=2)])
def test_ndg_and_third_order_fv_pass_validation(lib, kw):
    from paper_1709_01619_gb300 import _native
    cfg = _native.Config(**kw)
    h = ctypes.c_void_p()
    st = lib.cpr_init(ctypes.byref(cfg._c()), None, ctypes.byref(h))
    assert st in (_native.CPR_OK, _native.CPR_ECUDA)
    if st == _native.CPR_OK:
        lib.cpr_destroy(h)


def test_product_does_not_use_the_oracle():
    pkg = os.path.join(ROOT, "paper_1709_01619_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                with open(os.path.join(dirpath, f)) as fh:
                    src = fh.read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f
                assert "cpr_oracle" not in src and "liboracle" not in src, f


def test_context_needs_a_gpu():
    import torch
    from paper_1709_01619_gb300 import _native
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(RuntimeError):
        _native.Context(_native.Config())


def test_batch_init_rejects_unsupported_options(lib):
    from paper_1709_01619_gb300 import _native
    ok = _native.Config(eqn=1, nx=8, ny=8, p=2)
    bad = [
        _native.Config(eqn=1, nx=8, ny=8, p=2, limiter=1),
        _native.Config(eqn=1, nx=8, ny=8, p=2, dtype=1),
        _native.Config(eqn=1, nx=8, ny=8, p=2, pts=1),
        _native.Config(eqn=1, nx=8, ny=8, p=2, div=1),
        _native.Config(eqn=1, nx=0, ny=8, p=2),
    ]
    for b in bad:
        arr = (_native._Config * 2)(ok._c(), b._c())
        h = ctypes.c_void_p()
        assert lib.cpr_batch_init(arr, 2, None, ctypes.byref(h)) == _native.CPR_EINVAL
        assert not h.value and lib.cpr_batch_last_error(None)
    h = ctypes.c_void_p()
    assert lib.cpr_batch_init(None, 1, None, ctypes.byref(h)) == _native.CPR_EINVAL
    assert lib.cpr_batch_step(None, None, 1, 0.0, 0.0) == _native.CPR_EINVAL
    assert lib.cpr_batch_step_host(None, None, None, 1, 0.0, 0.0) == _native.CPR_EINVAL
    lib.cpr_batch_destroy(None)
