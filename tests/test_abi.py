"""The C ABI library loads and exports every entry point declared in
include/cf.h; argument validation that precedes any CUDA call works on a
machine without a GPU (CPU only, no compute calls)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cfmod():
    from paper_1406_6072_gb300 import _build
    _build.build()
    from paper_1406_6072_gb300 import cf
    return cf


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "cf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*CF_API\s+(?:const\s+)?\w+\*?\s+\**(cf_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("cf_embed", "cf_sample", "cf_sample_lp", "cf_lognormal_poisson", "cf_power_spectrum",
                     "cf_power_spectrum_counts", "cf_draw_noise", "cf_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(cfmod):
    lib = cfmod.raw_lib()
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_string(cfmod):
    assert "sm_103a" in cfmod.cf_version()
    assert isinstance(cfmod.cf_last_error(), str)


def test_argument_errors_before_any_cuda_call(cfmod):
    lib = cfmod.raw_lib()
    h = C.c_void_p()
    rep = cfmod.cf_embed_report()
    xi = cfmod.make_xi(cfmod.CF_XI_GAUSSIAN, 1.0, 2.0)
    assert lib.cf_embed(None, C.byref(xi), 0, None, C.byref(h), C.byref(rep)) == cfmod.CF_ERR_ARG
    g = cfmod.make_grid((3, 4), factor=3)  # embedding factors are 2, 4 or 8
    assert lib.cf_embed(C.byref(g), C.byref(xi), 0, None, C.byref(h), C.byref(rep)) == cfmod.CF_ERR_ARG
    assert "embed_factor" in cfmod.cf_last_error()
    g = cfmod.make_grid((4096, 4))  # 2n = 8192 too long
    assert lib.cf_embed(C.byref(g), C.byref(xi), 0, None, C.byref(h), C.byref(rep)) == cfmod.CF_ERR_UNSUPPORTED
    g = cfmod.make_grid((2049, 4))  # next power of two >= 2n is 8192
    assert lib.cf_embed(C.byref(g), C.byref(xi), 0, None, C.byref(h), C.byref(rep)) == cfmod.CF_ERR_UNSUPPORTED
    g = cfmod.make_grid((1024, 4), factor=8)
    assert lib.cf_embed(C.byref(g), C.byref(xi), 0, None, C.byref(h), C.byref(rep)) == cfmod.CF_ERR_UNSUPPORTED
    g4 = cfmod.make_grid((4, 4, 4, 4)[:3])
    g4.ndim = 4
    assert lib.cf_embed(C.byref(g4), C.byref(xi), 0, None, C.byref(h), C.byref(rep)) == cfmod.CF_ERR_ARG
    bad = cfmod.make_xi(cfmod.CF_XI_TABLE)
    g = cfmod.make_grid((4, 4))
    assert lib.cf_embed(C.byref(g), C.byref(bad), 0, None, C.byref(h), C.byref(rep)) == cfmod.CF_ERR_ARG
    assert lib.cf_sample(None, 0, 0, 1, cfmod.CF_F32, None, None, 0, None) == cfmod.CF_ERR_ARG
    assert lib.cf_draw_noise(0, 0, 1, 16, 3, cfmod.CF_F32, C.c_void_p(8), None) == cfmod.CF_ERR_ARG
    assert lib.cf_noise_selfcheck(None, None) == cfmod.CF_ERR_ARG
    assert lib.cf_draw_noise(0, 2**32 - 1, 2, 16, 4, cfmod.CF_F32, C.c_void_p(8), None) == cfmod.CF_ERR_ARG
    n = C.c_size_t()
    b = cfmod.make_bins(8)
    # any box: 1D, rectangular and non-power-of-two sides are accepted ...
    for shape in ((16,), (16, 32), (100, 60), (48, 80, 40)):
        gq = cfmod.make_grid(shape)
        assert lib.cf_power_spectrum_workspace_size(C.byref(gq), 4, C.byref(b), cfmod.CF_F32, C.byref(n)) == \
            cfmod.CF_OK
        assert n.value > 0
    # ... up to 2048 points for other lengths (Bluestein) and 4096 for powers of two
    for shape in ((3000, 16), (8192, 2)):
        gq = cfmod.make_grid(shape)
        assert lib.cf_power_spectrum_workspace_size(C.byref(gq), 4, C.byref(b), cfmod.CF_F32, C.byref(n)) == \
            cfmod.CF_ERR_UNSUPPORTED
    g4b = cfmod.make_grid((4, 4, 4))
    g4b.ndim = 4
    assert lib.cf_power_spectrum_workspace_size(C.byref(g4b), 4, C.byref(b), cfmod.CF_F32, C.byref(n)) == \
        cfmod.CF_ERR_ARG
    gs = cfmod.make_grid((16, 16))
    assert lib.cf_power_spectrum_workspace_size(C.byref(gs), 4, C.byref(b), cfmod.CF_F32, C.byref(n)) == cfmod.CF_OK
    assert n.value > 0
    b0 = cfmod.make_bins(0)
    assert lib.cf_power_spectrum_workspace_size(C.byref(gs), 4, C.byref(b0), cfmod.CF_F32, C.byref(n)) == \
        cfmod.CF_ERR_ARG
    blog = cfmod.make_bins(4, cfmod.CF_BINS_LOG, 0.0, 8.0)
    assert lib.cf_power_spectrum_workspace_size(C.byref(gs), 4, C.byref(blog), cfmod.CF_F32, C.byref(n)) == \
        cfmod.CF_ERR_ARG
    assert lib.cf_lognormal_poisson(None, 1, 4, 1, 1.0, 1.0, None, 0, 0, None, None, None) == cfmod.CF_ERR_ARG


def test_binding_does_not_import_the_oracle():
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r); import paper_1406_6072_gb300.cf; "
            "assert 'oracle' not in sys.modules; print('ok')" % ROOT)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    assert out.returncode == 0 and "ok" in out.stdout, out.stderr
