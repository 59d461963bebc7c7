"""Host-side checks of the C-ABI boundary that need no GPU: the library builds for sm_103a,
loads, exports every function include/fmbem.h declares, and rejects invalid input on the host
(mesh validation happens before any device work)."""
import numpy as np
import pytest

import fmbem_inputs as fi
import paper_1211_7177_gb300 as fm


def test_library_loads_and_exports_header():
    lib = fm.load_library()
    names = fm.header_functions()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_default_options():
    o = fm.fmbem_default_options()
    assert o.node_mode == fm.NODES_VERTEX and o.p == 8 and o.leaf_size == 64 and o.gmres_restart == 50
    assert o.solve_precision == fm.FP64 and o.profile_phases == 0


def _create(V, F, D, eps=(1.0, 2.25), mu=(1.0, 1.0), k0=1.0, **opt):
    return fm.fmbem_create(V, F, D, eps, mu, k0, fm.fmbem_default_options(**opt), stream=0)


@pytest.mark.parametrize("case", ["open", "flipped", "index", "domain", "degenerate", "junction"])
def test_invalid_meshes_rejected_on_host(case):
    V, F, D = fi.icosphere(1)
    F = F.copy()
    if case == "open":
        F = F[1:]
        D = D[1:]
    elif case == "flipped":
        F[3] = F[3][[0, 2, 1]]
    elif case == "index":
        F[0, 0] = len(V) + 5
    elif case == "domain":
        D = D.copy()
        D[0] = 7
    elif case == "degenerate":
        V = V.copy()
        a, b, c = F[5]
        V[c] = V[a] + 2.0 * (V[b] - V[a])        # collinear triangle
    elif case == "junction":
        D = D.copy()
        D[: len(D) // 2] = 2                      # one closed surface split between two scatterers
    eps = (1.0, 2.25, 3.0) if case in ("domain", "junction") else (1.0, 2.25)
    mu = (1.0, 1.0, 1.0) if case in ("domain", "junction") else (1.0, 1.0)
    if case == "domain":
        eps, mu = (1.0, 2.25), (1.0, 1.0)
        with pytest.raises(ValueError):
            _create(V, F, D, eps, mu)
        return
    with pytest.raises(fm.FMBEMError) as e:
        _create(V, F, D, eps, mu)
    assert e.value.status == 2, str(e.value)


def test_invalid_arguments_rejected():
    V, F, D = fi.icosphere(1)
    with pytest.raises(fm.FMBEMError) as e:
        _create(V, F, D, k0=-1.0)
    assert e.value.status == 1
    with pytest.raises(fm.FMBEMError) as e:
        _create(V, F, D, p=40)
    assert e.value.status == 1
    with pytest.raises(fm.FMBEMError) as e:
        _create(V, F, D, eps=(1.0, 0.0))
    assert e.value.status == 1


def test_boundary_option_and_null_handles_rejected():
    """The boundary option defaults to the penetrable formulation and an unknown value is refused
    before any device work; every entry point that takes a handle refuses NULL."""
    o = fm.fmbem_default_options()
    assert o.boundary == fm.PENETRABLE
    V, F, D = fi.icosphere(1)
    with pytest.raises(fm.FMBEMError) as e:
        _create(V, F, D, boundary=7)
    assert e.value.status == 1
    lib = fm.load_library()
    N = None
    z = np.zeros(3)
    zc = np.zeros(3, dtype=np.complex128)
    p3 = z.ctypes.data
    pc = zc.ctypes.data
    assert lib.fmbem_shape_gradient(N, 1, 1, 1, p3, pc, p3, pc, pc, None) == 1
    assert lib.fmbem_shape_gradient_near(N, 1, 1, 1, p3, pc, 1, p3, pc, None, pc, None) == 1
    assert lib.fmbem_interior_field(N, 1, 1, 1, p3, p3, pc, None, None) == 1
    assert lib.fmbem_near_field_fmm(N, 1, 1, 1, p3, None, None, pc, None, None) == 1
    assert lib.fmbem_near_field(N, 1, 1, 1, p3, None, None, pc, None, None) == 1
    assert lib.fmbem_matvec_host(N, pc, pc, 1, 0, 0, None) == 1


def test_injected_device_budget_fails_create_with_oom():
    """Fault injection on the host: with a device budget smaller than the first allocation,
    fmbem_create fails with FMBEM_ERR_OOM and a message naming the budget, after the mesh has
    been validated and before any device work."""
    V, F, D = fi.icosphere(1)
    lib = fm.load_library()
    lib.fmbem_debug_set_device_budget(0)
    try:
        with pytest.raises(fm.FMBEMError) as e:
            _create(V, F, D)
        assert e.value.status == 3 and "budget" in str(e.value)
    finally:
        lib.fmbem_debug_set_device_budget(-1)


def test_binding_declares_every_signature():
    """Every entry point declared in include/fmbem.h gets its ctypes signature (argument types)
    from the binding when the library is loaded, so scalars such as tolerances convert."""
    lib = fm.load_library()
    missing = [n for n in fm.header_functions() if getattr(lib, n).argtypes is None]
    assert not missing, missing


def test_header_is_plain_c_and_a_c_program_links(tmp_path):
    """include/fmbem.h compiles as C99 (no C++ types in the signatures), and a C program linked
    against the library runs the host-side entry points: default options, and the refusal of an
    open mesh before any device work."""
    import os
    import shutil
    import subprocess
    from paper_1211_7177_gb300 import build as b
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    fm.load_library()
    src = tmp_path / "use.c"
    src.write_text(r"""
#include <stdio.h>
#include "fmbem.h"
int main(void) {
    fmbem_options o;
    fmbem_default_options(&o);
    double V[12] = {0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1};
    int32_t F[9] = {0, 2, 1, 0, 1, 3, 0, 3, 2};   /* three faces of a tetrahedron: open */
    int32_t D[3] = {1, 1, 1};
    fmbem_mesh m = {4, V, 3, F, D, 1};
    fmbem_c64 eps[2] = {{1.0, 0.0}, {2.25, 0.0}}, mu[2] = {{1.0, 0.0}, {1.0, 0.0}};
    fmbem *h = NULL;
    fmbem_status st = fmbem_create(&m, eps, mu, 1.0, &o, NULL, &h);
    printf("%d %d %d %d %s\n", o.p, o.leaf_size, (int)st, h == NULL, fmbem_last_error(NULL));
    return 0;
}
""")
    exe = tmp_path / "use"
    libdir = os.path.dirname(b.LIB)
    include = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", include, str(src), "-o", str(exe), b.LIB,
                        "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    p, leaf, st, null, *msg = out.stdout.split(maxsplit=4)
    assert (p, leaf, st, null) == ("8", "64", "2", "1"), out.stdout


def test_near_singular_options_validated_before_device_work():
    """The near-singular correction is off by default (radius 0, the paper's one-point rule);
    a negative or non-finite radius and subdivision levels outside 0..6 are refused before any
    device work; fmbem_num_near_singular_pairs takes a NULL handle as zero pairs."""
    o = fm.fmbem_default_options()
    assert o.near_singular_radius == 0.0 and o.near_singular_levels == 3
    V, F, D = fi.icosphere(1)
    for kw in (dict(near_singular_radius=-1.0), dict(near_singular_radius=float("nan")),
               dict(near_singular_radius=1.5, near_singular_levels=7), dict(near_singular_levels=-1)):
        with pytest.raises(fm.FMBEMError) as e:
            _create(V, F, D, **kw)
        assert e.value.status == 1, kw
    assert fm.load_library().fmbem_num_near_singular_pairs(None) == 0


def test_fmm_tol_validated_before_device_work():
    o = fm.fmbem_default_options()
    assert o.fmm_tol == 0.0
    V, F, D = fi.icosphere(1)
    for bad in (-1e-5, 1.0, float("nan")):
        with pytest.raises(fm.FMBEMError) as e:
            _create(V, F, D, fmm_tol=bad)
        assert e.value.status == 1, bad


def test_adaptive_option_validated_before_device_work():
    """The octree is the paper's uniform tree by default; values other than 0 and 1 are refused
    before any device work."""
    o = fm.fmbem_default_options()
    assert o.adaptive == 0
    V, F, D = fi.icosphere(1)
    for bad in (-1, 2):
        with pytest.raises(fm.FMBEMError) as e:
            _create(V, F, D, adaptive=bad)
        assert e.value.status == 1, bad


def test_options_struct_layout_matches_the_header(tmp_path):
    """The binding's Options structure has the size and field offsets of the C fmbem_options
    (a C program prints them), so every option reaches the library as set."""
    import os
    import shutil
    import subprocess
    import ctypes
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    names = [n for n, _ in fm.Options._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"fmbem.h\"\nint main(void) {\n"
                   "    printf(\"%zu\\n\", sizeof(fmbem_options));\n" +
                   "".join(f"    printf(\"%zu\\n\", offsetof(fmbem_options, {n}));\n" for n in names) +
                   "    return 0;\n}\n")
    include = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    exe = tmp_path / "layout"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", include, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, timeout=60).stdout.split()]
    assert out[0] == ctypes.sizeof(fm.Options)
    assert out[1:] == [getattr(fm.Options, n).offset for n in names]
