"""The C-ABI library builds, loads without a GPU, exports every entry point the
headers declare, and rejects bad host arguments before touching the device."""
import ctypes
import glob
import os
import re

import pytest

from paper_2606_18314_b300 import build as cbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    cbuild.build()
    from paper_2606_18314_b300 import cert
    return cert.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(cert_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["cert_init", "cert_step", "cert_rebuild", "cert_allpairs", "cert_sync_result",
                     "cert_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_lists_every_symbol():
    from paper_2606_18314_b300 import cert
    assert set(declared_functions()) <= set(cert.EXPORTS)


def test_version_string(L):
    from paper_2606_18314_b300 import cert
    assert "sm_103a" in cert.cert_version()


def test_host_argument_validation_without_gpu(L):
    from paper_2606_18314_b300 import cert
    h = ctypes.c_void_p()
    # NULL config / NULL positions / bad dim are rejected before any CUDA call
    assert L.cert_init(ctypes.byref(h), None, None, None) == cert.CERT_EINVAL
    cfg = cert.cert_config()
    cfg.dim = 4
    cfg.n_scenes = 1
    cfg.n_total = 10
    assert L.cert_init(ctypes.byref(h), ctypes.byref(cfg), ctypes.c_void_p(16), None) == cert.CERT_EINVAL
    assert b"dim" in L.cert_last_error(None)
    cfg.dim = 3
    cfg.n_total = 2
    assert L.cert_init(ctypes.byref(h), ctypes.byref(cfg), ctypes.c_void_p(16), None) == cert.CERT_EINVAL
    cfg.n_total = 10
    cfg.audit = 8   # rho = 1, geometry = 2, cost = 4; other bits are rejected
    assert L.cert_init(ctypes.byref(h), ctypes.byref(cfg), ctypes.c_void_p(16), None) == cert.CERT_EINVAL
    assert b"audit" in L.cert_last_error(None)
    cfg.audit = 0
    cfg.frontier_rule = 3
    assert L.cert_init(ctypes.byref(h), ctypes.byref(cfg), ctypes.c_void_p(16), None) == cert.CERT_EINVAL
    assert b"frontier_rule" in L.cert_last_error(None)
    cfg.frontier_rule = 0
    cfg.bucket_factor = 3
    assert L.cert_init(ctypes.byref(h), ctypes.byref(cfg), ctypes.c_void_p(16), None) == cert.CERT_EINVAL
    cfg.bucket_factor = 0
    cfg.cell_quantile = 1.5
    assert L.cert_init(ctypes.byref(h), ctypes.byref(cfg), ctypes.c_void_p(16), None) == cert.CERT_EINVAL
    cfg.cell_quantile = 0.0
    cfg.policy = 3
    assert L.cert_init(ctypes.byref(h), ctypes.byref(cfg), ctypes.c_void_p(16), None) == cert.CERT_EINVAL
    assert L.cert_step(None, None, ctypes.c_float(1e-3), 1, None, None) == cert.CERT_EINVAL
    assert L.cert_allpairs(None, 10, 3, None, 0, None, None, None, None) == cert.CERT_EINVAL
    assert L.cert_allpairs(ctypes.c_void_p(16), 2, 3, None, 0, ctypes.c_void_p(16), ctypes.c_void_p(16),
                           ctypes.c_void_p(16), None) == cert.CERT_EINVAL
    assert L.cert_sync_result(None, None) == cert.CERT_EINVAL


def test_struct_layouts_match_header():
    from paper_2606_18314_b300 import cert
    # cert_scene_result: 2 doubles + 18 four-byte fields + 2 doubles + 2 uint64 cycle counts
    assert ctypes.sizeof(cert.cert_scene_result) == 16 + 18 * 4 + 16 + 16
    assert ctypes.sizeof(cert.cert_config) == 4 + 4 + 8 + 8 + 4 + 4 + 16


def test_python_modules_import_without_gpu():
    import importlib
    for name in ["paper_2606_18314_b300.cert", "paper_2606_18314_b300.selector", "paper_2606_18314_b300.scenes",
                 "paper_2606_18314_b300.build"]:
        importlib.import_module(name)
    from paper_2606_18314_b300 import selector
    p = selector.he_init(0)
    assert p.shape == (4866,) and p.dtype.name == "float32"
    assert abs(float(p[:512].std()) - (2.0 / 8) ** 0.5) < 0.1     # He-normal fan-in 8
    assert float(abs(p[512:576]).max()) == 0.0                       # zero biases


def test_knn_rejects_bad_arguments_without_a_gpu(L):
    from paper_2606_18314_b300 import cert
    h = ctypes.c_void_p()
    cfg = cert.cert_knn_config()
    cfg.dim, cfg.k, cfg.n = 3, 4, 100

    def init():
        return L.cert_knn_init(ctypes.byref(h), ctypes.byref(cfg), ctypes.c_void_p(16), None)

    for field, bad, good, word in [("dim", 4, 3, b"dim"), ("k", 0, 4, b"k must"), ("k", 17, 4, b"k must"),
                                   ("n", 5, 100, b"n must"), ("cell_scale", -1.0, 0.0, b"cell_scale"),
                                   ("cell_scale", float("inf"), 0.0, b"cell_scale"), ("reserved", 1, 0, b"reserved")]:
        setattr(cfg, field, bad)
        assert init() == cert.CERT_EINVAL, field
        assert word in L.cert_last_error(None), field
        assert h.value is None
        setattr(cfg, field, good)
    assert L.cert_knn_init(ctypes.byref(h), ctypes.byref(cfg), None, None) == cert.CERT_EINVAL
    assert L.cert_knn_step(None, ctypes.c_void_p(16), ctypes.c_float(1e-3), 1, None) == cert.CERT_EINVAL
    assert L.cert_knn_sync_result(None, None) == cert.CERT_EINVAL
    assert L.cert_knn_get_views(None, None) == cert.CERT_EINVAL
    L.cert_knn_destroy(None)
    assert ctypes.sizeof(cert.cert_knn_config) == 24
    assert ctypes.sizeof(cert.cert_knn_result) == 40
    assert ctypes.sizeof(cert.cert_knn_views) == 5 * 8 + 8 + 4 + 4


def test_debug_variant_loads_and_exports_every_symbol():
    """libcert_debug.so (index-checked kernels) is selected by CERT_LIB_VARIANT=debug
    and exports the same boundary."""
    import subprocess
    import sys
    cbuild.build(debug=True)
    code = ("from paper_2606_18314_b300 import cert; L = cert.lib(); "
            "assert cert.LIB_PATH.endswith('libcert_debug.so'); "
            "missing = [n for n in cert.EXPORTS if not hasattr(L, n)]; assert not missing, missing; print('ok')")
    env = dict(os.environ, CERT_LIB_VARIANT="debug")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and "ok" in out.stdout, out.stderr[-2000:]


def test_source_fingerprints_match_the_build(L):
    """The library reports the fingerprint of the sources it was built from,
    unit by unit, so a profiler measurement can name the build it belongs to."""
    from paper_2606_18314_b300 import cert
    fps = cbuild.fingerprints()
    assert "step_kernels" in fps and "allpairs" in fps
    for unit, fp in fps.items():
        assert cert.cert_source_fingerprint(unit) == fp, unit
    assert cert.cert_source_fingerprint("no_such_unit") is None
