"""CPU checks: libflood.so loads and exports every entry point of include/flood.h,
and the host-side input preparation (complex builder, generators) is sound."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2509_22432_b300 import complex_from_simplices, data, delaunay_complex
from paper_2509_22432_b300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "flood.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(flood_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = _lib.get()
    declared = _declared_functions()
    assert len(declared) >= 9
    for name in declared:
        assert hasattr(lib, name), name
        assert name in _lib.exported_symbols(), name
    assert lib.flood_version().decode() == "0.1.0"


def test_library_is_the_in_tree_build():
    lib = _lib.get()
    assert os.path.dirname(os.path.abspath(lib._name)) == os.path.join(ROOT, "paper_2509_22432_b300")


def test_status_codes_match_header():
    text = open(os.path.join(ROOT, "include", "flood.h")).read()
    for code, name in _lib.STATUS.items():
        assert re.search(rf"{name}\s*=\s*{code}\b", text), name


def test_delaunay_complex_is_closed_with_consistent_facets():
    X = data.shape_mix_cloud(5000, seed=1)
    cx = delaunay_complex(X[:200])
    for k in range(1, 4):
        S = cx.simplices[k]
        assert np.all(np.diff(S, axis=1) > 0)                     # ascending ids
        keys = [tuple(r) for r in S]
        assert keys == sorted(keys)                               # lexicographic rows
        for j in range(k + 1):
            face = np.delete(S, j, axis=1)
            assert np.array_equal(cx.simplices[k - 1][cx.facets[k][:, j]], face)
    # Euler characteristic of a triangulated 3-ball: V - E + F - T = 1
    n = cx.counts
    assert n[0] - n[1] + n[2] - n[3] == 1


def test_complex_from_simplices_handles_lower_dims():
    cx = complex_from_simplices([np.array([[0, 1, 2]]), np.array([[2, 3]])], 4)
    assert cx.counts == [4, 4, 1]
    assert np.array_equal(cx.simplices[1], [[0, 1], [0, 2], [1, 2], [2, 3]])


def test_generators_are_seeded_float32_and_shaped():
    for f, n in ((data.sphere_cloud, 1000), (data.torus_cloud, 1000), (data.shape_mix_cloud, 2000),
                 (data.swisscheese_cloud, 1000)):
        a, b = f(n), f(n)
        assert a.dtype == np.float32 and a.shape == (n, 3)
        assert np.array_equal(a, b)
    t = data.torus_cloud(20000, noise=0.0)
    rho = np.sqrt(t[:, 0].astype(np.float64) ** 2 + t[:, 1] ** 2)
    assert np.allclose((rho - 1.0) ** 2 + t[:, 2].astype(np.float64) ** 2, 0.09, atol=1e-5)
    s = data.serving_sizes()
    assert s.min() >= 2000 and s.max() <= 200000 and len(s) == 512


def test_new_entry_points_reject_bad_arguments_before_any_device_call():
    """Host-side validation of the given-sets, masked, faces and backward entry points."""
    import ctypes as C
    lib = _lib.get()
    P4, I64x4, I32x4 = _lib.P4, _lib.I64x4, _lib.I32x4
    null4, n4 = P4(), I64x4(0, 3, 3, 1)
    einval = -1
    # faces: negative count, NULL count outputs
    n2, n1 = C.c_int64(0), C.c_int64(0)
    assert lib.flood_complex_faces(None, -1, 4, None, None, None, None, None, C.byref(n2), C.byref(n1), None) == einval
    assert lib.flood_complex_faces(None, 1, 4, None, None, None, None, None, None, None, None) == einval
    assert lib.flood_complex_faces(None, 1, 1 << 21, None, None, None, None, None, C.byref(n2), C.byref(n1),
                                   None) == einval
    # empty input succeeds without touching the device
    assert lib.flood_complex_faces(None, 0, 4, None, None, None, None, None, C.byref(n2), C.byref(n1), None) == 0
    assert n2.value == 0 and n1.value == 0
    # given sets, masked comparator, given backward: a NULL grid is rejected on the host
    assert lib.flood_filtration_given(None, None, 4, null4, null4, n4, P4(), I32x4(), null4, null4, None) == einval
    assert lib.flood_filtration_masked(None, None, 4, null4, n4, 6, null4, None, None) == einval
    assert lib.flood_filtration_given_backward(None, None, 4, null4, n4, P4(), I32x4(), null4, null4, None, None,
                                               None) == einval
    assert lib.flood_last_error().decode() != ""


def test_planar_delaunay_complex():
    """Ambient dimension 2: a triangulated disk (Euler characteristic 1), z = 0 required."""
    X = data.annulus_cloud(3000, seed=3)
    cx = delaunay_complex(X[:200], dim=2)
    assert len(cx.counts) == 3
    assert cx.counts[0] - cx.counts[1] + cx.counts[2] == 1
    assert np.all(np.diff(cx.simplices[2], axis=1) > 0)
    Y = X[:50].copy()
    Y[0, 2] = 1e-3
    with pytest.raises(ValueError):
        delaunay_complex(Y, dim=2)


def test_header_is_plain_c():
    """include/flood.h compiles as C99 (pedantic) and as C++: the boundary carries no torch or
    C++ types."""
    import shutil
    import subprocess
    import tempfile
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "use.c")
        with open(src, "w") as f:
            f.write('#include "flood.h"\nint main(void) { return flood_version() ? 0 : 1; }\n')
        r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                            "-I", os.path.join(ROOT, "include"), src], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_noalloc_fixed_array_holds_fps_scratch_at_its_maximum_size():
    """flood_fps_noalloc's fixed array (27 MiB) must hold FPS's scratch for 2^20 points at any
    launch width; the largest need is the streamed kernel (one block), which adds 4 bytes of
    running minimum per point."""
    from paper_2509_22432_b300 import ops

    worst = ops.fps_scratch_bytes(1 << 20, 1)
    assert worst >= (16 + 4 + 4) << 20                    # point copy, running minima, Morton codes
    assert worst <= 27 << 20, worst
    assert ops.fps_scratch_bytes(1000, 1) < ops.fps_scratch_bytes(100_000, 1)
