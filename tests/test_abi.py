"""The C-ABI library builds for sm_103a, loads, and exports every function include/sc.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import subprocess

from paper_2410_21207_gb300 import binding, build


def test_header_declares_the_boundary():
    names = binding.header_functions()
    for required in ("sc_energy", "sc_find_seam", "sc_carve", "sc_carve_batch", "sc_check"):
        assert required in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in binding.header_functions():
        assert hasattr(lib, name), name
    # plain C names (extern "C"), no C++ mangling
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    for name in binding.header_functions():
        assert name in exported, name


def test_version_and_error_string_without_gpu():
    lib = binding.load()
    assert lib.sc_version() >= 100
    assert isinstance(lib.sc_last_error(), bytes)


def test_argument_errors_are_synchronous():
    """Bad arguments are rejected before any CUDA call, so they work on a machine without a GPU."""
    lib = binding.load()
    P = ctypes.c_void_p
    fake = P(0x1000)
    # null pointers
    assert lib.sc_carve(P(0), 10, 10, 3, 5, 5, fake, P(0), P(0), P(0)) == binding.SC_EINVAL
    # enlargement
    assert lib.sc_carve(fake, 10, 10, 3, 11, 10, fake, P(0), P(0), P(0)) == binding.SC_EINVAL
    assert b"enlargement" in lib.sc_last_error()
    # channel count
    assert lib.sc_carve(fake, 10, 10, 2, 5, 5, fake, P(0), P(0), P(0)) == binding.SC_EINVAL
    # zero target
    assert lib.sc_carve_plain(fake, 10, 10, 3, 0, 5, fake, P(0), P(0), P(0)) == binding.SC_EINVAL
    # size limits
    assert lib.sc_carve(fake, binding.MAX_ROWS + 1, 10, 3, 5, 5, fake, P(0), P(0), P(0)) == binding.SC_EINVAL
    assert lib.sc_find_seam(fake, 0, 10, fake, P(0), P(0)) == binding.SC_EINVAL
    assert lib.sc_find_seam(fake, 10, binding.MAX_COLS + 1, fake, P(0), P(0)) == binding.SC_EINVAL
    assert lib.sc_energy(fake, 10, 10, 5, fake, P(0)) == binding.SC_EINVAL
    assert lib.sc_carve_batch(P(0), 0, P(0)) == binding.SC_EINVAL
    assert lib.sc_enlarge(fake, 10, 10, 3, 10, fake, P(0), P(0)) == binding.SC_EINVAL   # k = 0
    assert lib.sc_enlarge(fake, 10, 10, 3, 20, fake, P(0), P(0)) == binding.SC_EINVAL   # k = W
    assert lib.sc_enlarge(P(0), 10, 10, 3, 15, fake, P(0), P(0)) == binding.SC_EINVAL
    assert lib.sc_greedy_seam(P(0), 10, 10, fake, P(0), P(0)) == binding.SC_EINVAL
    assert lib.sc_selftest_wait_timeout(0, P(0)) == binding.SC_EINVAL
    assert lib.sc_find_seam_static(P(0), 10, 10, fake, P(0), P(0)) == binding.SC_EINVAL
    assert lib.sc_find_seam_static(fake, 10, binding.MAX_COLS + 1, fake, P(0), P(0)) == binding.SC_EINVAL
    # a map larger than the static scratch array is refused before any CUDA call, with the bytes named
    assert lib.sc_find_seam_static(fake, 4000, 4000, fake, P(0), P(0)) == binding.SC_EINVAL
    assert b"bytes of scratch" in lib.sc_last_error()
    assert lib.sc_find_seam_static_selftest(0, 10, fake, P(0), P(0)) == binding.SC_EINVAL
    g = ctypes.c_double(0.0)
    assert lib.sc_probe_copy_bandwidth(ctypes.c_size_t(100), 1, ctypes.byref(g)) == binding.SC_EINVAL
    assert lib.sc_probe_copy_bandwidth(ctypes.c_size_t(1 << 20), 0, ctypes.byref(g)) == binding.SC_EINVAL
    assert lib.sc_find_seam_static_selftest(1000, 0, fake, P(0), P(0)) == binding.SC_EINVAL
    assert lib.sc_find_seam_multi_shape(5, 8) == binding.SC_EINVAL
    assert lib.sc_find_seam_multi_shape(0, 0) == binding.SC_OK
    maps = (P * 2)(fake, P(0))
    assert lib.sc_find_seam_multi(maps, 0, 10, 10, fake, P(0), P(0)) == binding.SC_EINVAL
    assert lib.sc_find_seam_multi(maps, 2, 10, 10, fake, P(0), P(0)) == binding.SC_EINVAL   # null map
    assert lib.sc_find_seam_multi(maps, 1, 10, binding.MAX_COLS + 1, fake, P(0), P(0)) == binding.SC_EINVAL
