"""Host-side checks of the C ABI (no GPU needed): the library builds for sm_103a, loads, exports
every function include/evp.h declares, and the pure-host entry points validate their inputs."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "evp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:int|void|char)\s*\*?\s*(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1509_04953_gb300 import build
    build.build()
    from paper_1509_04953_gb300 import evp
    return evp.load()


def test_header_declares_the_boundary():
    fns = header_functions()
    for name in ("evp_init", "evp_increment", "drx_nucleate", "pf_step", "get_fields", "set_fields",
                 "evp_destroy", "evp_last_error", "evp_workspace_bytes", "evp_voronoi", "evp_rfft3d"):
        assert name in fns


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_binding_declares_argument_types_for_every_symbol(lib):
    """The Python binding gives every declared function its argument and result types, so that ctypes never
    passes a device pointer or a size through its default 32-bit int conversion."""
    for name in header_functions():
        fn = getattr(lib, name)
        assert fn.argtypes is not None, name
        assert fn.restype is not None or name == "evp_destroy", name


def test_workspace_bytes_validates_config(lib):
    from paper_1509_04953_gb300 import evp
    cfg = evp.make_config(16, 8)
    nb = C.c_size_t(0)
    assert lib.evp_workspace_bytes(C.byref(cfg), C.byref(nb)) == 0
    n16 = nb.value
    assert n16 > 16 ** 3 * 8 * 60
    cfg32 = evp.make_config(32, 8)
    assert lib.evp_workspace_bytes(C.byref(cfg32), C.byref(nb)) == 0
    assert 6 < nb.value / n16 < 10
    cfgm = evp.make_config(32, 8, precision="mixed")
    nbm = C.c_size_t(0)
    assert lib.evp_workspace_bytes(C.byref(cfgm), C.byref(nbm)) == 0 and nbm.value < nb.value
    for bad in (dict(n=12), dict(n=2), dict(n=512), dict(kmax=9), dict(kmax=0), dict(grains=0),
                dict(max_iter=0), dict(newton_tol=0.0), dict(precision="x")):
        kw = dict(n=16, grains=8)
        kw.update(bad)
        if kw.get("precision") == "x":
            c = evp.make_config(16, 8)
            c.precision = 7
        else:
            c = evp.make_config(**kw)
        assert lib.evp_workspace_bytes(C.byref(c), C.byref(nb)) == -1


def test_workspace_bytes_validates_solver_and_law_options(lib):
    """The scheme, law, reference-medium and Newton-mode fields are checked on the host: out-of-range values
    and combinations the library does not implement return EVP_ERR_ARG with a reason; valid ones are accepted."""
    import math
    from paper_1509_04953_gb300 import evp
    nb = C.c_size_t(0)

    def rc_of(**kw):
        fields = {k: kw.pop(k) for k in list(kw) if k in ("law_code", "newton_code", "scheme_code")}
        c = evp.make_config(16, 8, **kw)
        if "law_code" in fields:
            c.law = fields["law_code"]
        if "newton_code" in fields:
            c.newton_mode = fields["newton_code"]
        if "scheme_code" in fields:
            c.scheme = fields["scheme_code"]
        return lib.evp_workspace_bytes(C.byref(c), C.byref(nb))

    for ok in (dict(law="mr"), dict(law="mr", scheme="al", al_scale=8.0), dict(ref_scale=0.0), dict(ref_scale=0.5),
               dict(ref_scale=1.3), dict(ref_scale=4.0), dict(scheme="al", al_scale=1.0), dict(pf_refine=2),
               dict(precision="mixed", newton="reuse", newton_adapt=0.0)):
        assert rc_of(**ok) == 0, ok
    for bad in (dict(law_code=2), dict(law_code=-1), dict(ref_scale=0.49), dict(ref_scale=4.01),
                dict(ref_scale=-1.0), dict(ref_scale=math.nan), dict(scheme_code=2), dict(scheme="al", al_scale=0.5),
                dict(scheme="al", al_scale=math.nan), dict(pf_refine=3), dict(pf_refine=-1), dict(newton_adapt=-0.1),
                dict(newton_code=3),
                dict(law="mr", precision="fp64", newton="f32_tangent"),      # FP32 tangent: power law only
                dict(precision="mixed", newton="f32_tangent")):              # FP32 tangent: FP64 path only
        assert rc_of(**bad) == -1, bad


def test_init_rejects_bad_arguments_before_touching_the_device(lib):
    """Argument errors are returned (with a reason) before any CUDA call is made."""
    import numpy as np
    from paper_1509_04953_gb300 import evp, synth
    cfg = evp.make_config(16, 8)
    p = evp.make_params(synth.Material())
    h = C.c_void_p()
    g = np.zeros(16 ** 3, dtype=np.int32)
    q = np.zeros(32)
    # NULL workspace
    rc = lib.evp_init(C.byref(h), C.byref(cfg), C.byref(p), g.ctypes.data, q.ctypes.data, 1, None, 0, None)
    assert rc == -1 and b"NULL" in lib.evp_last_error(h)
    lib.evp_destroy(h)
    # workspace too small (a fake, never dereferenced address)
    h = C.c_void_p()
    rc = lib.evp_init(C.byref(h), C.byref(cfg), C.byref(p), g.ctypes.data, q.ctypes.data, 1, 1 << 20, 1024, None)
    assert rc == -6 and b"workspace" in lib.evp_last_error(h)
    lib.evp_destroy(h)


def test_build_entry_point_compiles_everything():
    import importlib
    ge = importlib.import_module("__graft_entry__")
    ge.build()
    assert os.path.exists(os.path.join(ROOT, "paper_1509_04953_gb300", "libevp_gb300.so"))
    assert os.path.exists(os.path.join(ROOT, "oracle", "liboracle.so"))


def test_product_path_fails_loudly_without_a_gpu():
    """No CPU fallback: without a CUDA device every entry of the binding that would compute raises."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import numpy as np
    from paper_1509_04953_gb300 import evp, synth
    n, G = 8, 2
    g0 = np.zeros(n ** 3, dtype=np.int32)
    with pytest.raises(evp.EVPError, match="no CUDA device"):
        evp.Solver(n, G, g0, synth.orientations(G, 0), synth.Material(), 0)
    x = torch.zeros((1, n, n, n), dtype=torch.float64)
    for call in (lambda: evp.rfft3d(x), lambda: evp.stress_residual(torch.zeros((6, n, n, n))),
                 lambda: evp.voronoi(n, synth.voronoi_seeds(n, G, 0))):
        with pytest.raises(evp.EVPError, match="no CUDA device"):
            call()


def test_residual_partials_fit_the_allocation_free_array_at_every_size(lib):
    """evp_stress_residual_noalloc keeps the z pass's per-block partial sums in a fixed array of 8192 doubles.
    The scratch that evp_stress_residual asks of its caller holds exactly those partial sums, so it must fit in
    the fixed array for every size the allocation-free entry point accepts (n <= 256, every precision); the
    largest, n = 256 in FP64, fills it exactly."""
    nb = C.c_size_t(0)
    sizes = {}
    for prec in (0, 1, 2):
        for n in (4, 8, 16, 32, 64, 128, 256):
            assert lib.evp_residual_scratch_bytes(n, prec, C.byref(nb)) == 0
            assert 0 < nb.value <= 8192 * 8, (n, prec, nb.value)
            sizes[(n, prec)] = nb.value
    assert max(sizes.values()) == 8192 * 8
