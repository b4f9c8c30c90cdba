"""The C-ABI library loads, exports every symbol include/scd.h declares, and rejects bad
arguments synchronously (these checks run before any CUDA call, so no GPU is needed)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2506_18003_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "scd.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(scd_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_what_binding_declares():
    assert declared_functions() == sorted(binding.SIGNATURES)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_library_hides_internal_symbols():
    out = os.popen(f"nm -D --defined-only {binding.LIB_PATH}").read()
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    ours = {s for s in exported if s.startswith("scd")}
    assert ours == set(declared_functions())


def test_status_strings(lib):
    for s in range(7):
        assert lib.scd_status_string(s)
    assert lib.scd_version() >= 100


def test_workspace_queries(lib):
    assert lib.scd_fam_workspace_bytes(65728, 256, 64, 1024, 0) == 2 * 256 * 1024 * 8 + 2048   # X, Y, norm
    assert lib.scd_ssca_workspace_bytes(1 << 20, 256, 0) >= 256 * (1 << 20) * 8
    assert lib.scd_fam_workspace_bytes(280, 32, 8, 32, 0) % 256 == 0
    # a length that is not a power of two: two channel rows of the 2^14-point cyclic transform
    assert lib.scd_ssca_workspace_bytes(5000, 32, 0) >= 2 * 32 * (1 << 14) * 8


FAKE = ctypes.c_void_p(1 << 20)        # aligned, never dereferenced: validation fails first


@pytest.mark.parametrize("N,Np,L,P,expect", [
    (280, 32, 8, 32, None),                            # valid (not run here)
    (279, 32, 8, 32, binding.SCD_ERR_ARG),             # N < (P-1) L + Np
    (280, 32, 0, 32, binding.SCD_ERR_ARG),             # L < 1
    (280, 24, 8, 32, binding.SCD_ERR_UNSUPPORTED),     # Np not a power of two
    (280, 8, 8, 32, binding.SCD_ERR_UNSUPPORTED),      # Np below 16
    (4000, 512, 8, 32, binding.SCD_ERR_UNSUPPORTED),   # Np above 256
    (280, 32, 8, 30, binding.SCD_ERR_WORKSPACE),       # P not a power of two: accepted (no workspace given)
    (1 << 20, 32, 1, 8193, binding.SCD_ERR_UNSUPPORTED),   # above 8192 and not a power of two
    (1 << 20, 32, 1, 32768, binding.SCD_ERR_UNSUPPORTED),
])
def test_fam_argument_validation(lib, N, Np, L, P, expect):
    if expect is None:
        return
    assert lib.scd_fam(FAKE, N, Np, L, P, None, FAKE, None) == expect


def test_null_and_misaligned_pointers(lib):
    assert lib.scd_fam(None, 280, 32, 8, 32, None, FAKE, None) == binding.SCD_ERR_ARG
    assert lib.scd_fam(FAKE, 280, 32, 8, 32, None, None, None) == binding.SCD_ERR_ARG
    assert lib.scd_fam(ctypes.c_void_p((1 << 20) + 4), 280, 32, 8, 32, None, FAKE, None) == binding.SCD_ERR_ARG
    assert lib.scd_fam(FAKE, 280, 32, 8, 32, None, ctypes.c_void_p((1 << 20) + 8), None) == binding.SCD_ERR_ARG
    assert lib.scd_ssca(None, 4096, 32, None, FAKE, None) == binding.SCD_ERR_ARG
    assert lib.scd_fam_map(None, 32, 8, 32, FAKE, None) == binding.SCD_ERR_ARG
    assert lib.scd_ssca_map(FAKE, 4096, 32, None, None) == binding.SCD_ERR_ARG


@pytest.mark.parametrize("N,Np,expect", [
    (2048, 32, binding.SCD_ERR_UNSUPPORTED),           # below 2^12
    (1 << 21, 32, binding.SCD_ERR_UNSUPPORTED),        # above 2^20
    (5000, 32, binding.SCD_ERR_WORKSPACE),             # not a power of two: accepted (no workspace given)
    (4095, 32, binding.SCD_ERR_UNSUPPORTED),           # below 2^12
    ((1 << 19) + 1, 32, binding.SCD_ERR_UNSUPPORTED),  # above 2^19 and not a power of two
    (4096, 48, binding.SCD_ERR_UNSUPPORTED),
])
def test_ssca_argument_validation(lib, N, Np, expect):
    assert lib.scd_ssca(FAKE, N, Np, None, FAKE, None) == expect


def test_workspace_is_required(lib):
    o = binding.ScdOpts()
    o.precision = 0
    o.map_power = 1
    assert lib.scd_fam(FAKE, 280, 32, 8, 32, None, FAKE, ctypes.byref(o)) == binding.SCD_ERR_WORKSPACE
    o.workspace = 1 << 20
    o.workspace_bytes = 16
    assert lib.scd_ssca(FAKE, 4096, 32, None, FAKE, ctypes.byref(o)) == binding.SCD_ERR_WORKSPACE


def test_map_validation(lib):
    o = binding.ScdOpts()
    o.map_power = 3
    assert lib.scd_fam_map(FAKE, 32, 8, 32, FAKE, ctypes.byref(o)) == binding.SCD_ERR_ARG
    assert lib.scd_fam_map(FAKE, 32, 20, 32, FAKE, None) == binding.SCD_ERR_UNSUPPORTED   # 2L > Np
    assert lib.scd_fam_map(FAKE, 32, 3, 8, FAKE, None) == binding.SCD_ERR_UNSUPPORTED     # PL % Np


def test_variant_validation(lib):
    o = binding.ScdOpts()
    o.map_power = 1
    o.workspace = 1 << 20
    o.workspace_bytes = 1 << 40
    o.y = (1 << 20) + 4                                  # misaligned second signal
    assert lib.scd_fam(FAKE, 280, 32, 8, 32, None, FAKE, ctypes.byref(o)) == binding.SCD_ERR_ARG
    assert lib.scd_ssca(FAKE, 4096, 32, None, FAKE, ctypes.byref(o)) == binding.SCD_ERR_ARG
    o.y = None
    o.conjugate = 2                                      # not 0 / 1
    assert lib.scd_fam(FAKE, 280, 32, 8, 32, None, FAKE, ctypes.byref(o)) == binding.SCD_ERR_ARG
    assert lib.scd_ssca(FAKE, 4096, 32, None, FAKE, ctypes.byref(o)) == binding.SCD_ERR_ARG
    o.conjugate = 1
    assert lib.scd_fam_noalloc(FAKE, 280, 32, 8, 32, None, FAKE, ctypes.byref(o)) == binding.SCD_ERR_UNSUPPORTED
    o.conjugate = 0
    o.y = 1 << 20                                        # host variants take no second signal
    assert lib.scd_fam_host(FAKE, 280, 32, 8, 32, None, FAKE, ctypes.byref(o)) == binding.SCD_ERR_ARG
    assert lib.scd_ssca_host(FAKE, 4096, 32, None, FAKE, ctypes.byref(o)) == binding.SCD_ERR_ARG


def test_profile_validation(lib):
    assert lib.scd_fam_alpha_profile(None, 32, 8, 32, FAKE, None) == binding.SCD_ERR_ARG
    assert lib.scd_fam_alpha_profile(FAKE, 32, 20, 32, FAKE, None) == binding.SCD_ERR_UNSUPPORTED
    assert lib.scd_ssca_alpha_profile(FAKE, 4096, 32, None, None) == binding.SCD_ERR_ARG
    assert lib.scd_ssca_alpha_profile(FAKE, 5000, 32, FAKE, None) == binding.SCD_ERR_UNSUPPORTED
    o = binding.ScdOpts()
    o.map_power = 0
    assert lib.scd_ssca_alpha_profile(FAKE, 4096, 32, FAKE, ctypes.byref(o)) == binding.SCD_ERR_ARG


def test_opts_layout_matches_header(tmp_path):
    """The ctypes mirror of scd_opts has the C struct's size and field offsets (a C
    program compiled against include/scd.h prints them)."""
    fields = [f for f, _ in binding.ScdOpts._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"scd.h\"\nint main(void) {\n"
                   + f'  printf("%zu\\n", sizeof(scd_opts));\n'
                   + "".join(f'  printf("%zu\\n", offsetof(scd_opts, {f}));\n' for f in fields)
                   + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(binding.ScdOpts)] + [getattr(binding.ScdOpts, f).offset for f in fields]
    assert got == want


def test_stream_plan_validation(lib):
    h = ctypes.c_void_p()
    assert lib.scd_stream_plan_create(1, 4096, 0, 4, 32, 1, 0, ctypes.byref(h)) == binding.SCD_ERR_ARG   # hop 0
    assert lib.scd_stream_plan_create(1, 4096, 1024, 0, 32, 1, 0, ctypes.byref(h)) == binding.SCD_ERR_ARG  # no window
    # the kept overlap (W - hop = 3072) would overlap its own source (nwin * hop = 2048)
    assert lib.scd_stream_plan_create(1, 4096, 1024, 2, 32, 1, 0, ctypes.byref(h)) == binding.SCD_ERR_ARG
    assert lib.scd_stream_advance(None, FAKE, FAKE, 0, None) == binding.SCD_ERR_ARG


def test_chebyshev_window_validation(lib):
    assert lib.scd_chebyshev_window(1, 100.0, FAKE, None) == binding.SCD_ERR_ARG
    assert lib.scd_chebyshev_window(257, 100.0, FAKE, None) == binding.SCD_ERR_ARG
    assert lib.scd_chebyshev_window(64, 0.0, FAKE, None) == binding.SCD_ERR_ARG
    assert lib.scd_chebyshev_window(64, float("nan"), FAKE, None) == binding.SCD_ERR_ARG
    assert lib.scd_chebyshev_window(64, 100.0, None, None) == binding.SCD_ERR_ARG


def test_host_fault_injection(lib, monkeypatch):
    """SCD_FAULT_INJECT=host:<site> makes that entry point fail after its argument checks and
    before any GPU work, with a message naming the site (no GPU needed)."""
    o = binding.ScdOpts()
    o.map_power = 1
    o.workspace = 1 << 20
    o.workspace_bytes = 1 << 40
    monkeypatch.setenv("SCD_FAULT_INJECT", "host:fam")
    assert lib.scd_fam(FAKE, 280, 32, 8, 32, None, FAKE, ctypes.byref(o)) == binding.SCD_ERR_CUDA
    assert b"injected fault at fam" in lib.scd_last_error()
    # argument errors still come first
    assert lib.scd_fam(FAKE, 279, 32, 8, 32, None, FAKE, ctypes.byref(o)) == binding.SCD_ERR_ARG
    monkeypatch.setenv("SCD_FAULT_INJECT", "host:ssca")
    assert lib.scd_ssca(FAKE, 4096, 32, None, FAKE, ctypes.byref(o)) == binding.SCD_ERR_CUDA
    monkeypatch.setenv("SCD_FAULT_INJECT", "host:ssca_map")
    assert lib.scd_ssca_map(FAKE, 4096, 32, FAKE, None) == binding.SCD_ERR_CUDA
    monkeypatch.setenv("SCD_FAULT_INJECT", "host:fam_map")
    assert lib.scd_fam_map(FAKE, 32, 8, 32, FAKE, None) == binding.SCD_ERR_CUDA
    monkeypatch.delenv("SCD_FAULT_INJECT")
    assert lib.scd_fam_map(None, 32, 8, 32, FAKE, None) == binding.SCD_ERR_ARG


def test_normalise_validation(lib):
    o = binding.ScdOpts()
    o.map_power = 1
    o.workspace = 1 << 20
    o.workspace_bytes = 1 << 40
    o.normalise = 3
    assert lib.scd_fam(FAKE, 280, 32, 8, 32, None, FAKE, ctypes.byref(o)) == binding.SCD_ERR_ARG
    o.normalise = 1
    o.y = 1 << 20                                        # cross estimate: not defined
    assert lib.scd_fam(FAKE, 280, 32, 8, 32, None, FAKE, ctypes.byref(o)) == binding.SCD_ERR_UNSUPPORTED
    assert lib.scd_ssca(FAKE, 4096, 32, None, FAKE, ctypes.byref(o)) == binding.SCD_ERR_UNSUPPORTED
    o.y = None
    assert lib.scd_fam_noalloc(FAKE, 280, 32, 8, 32, None, FAKE, ctypes.byref(o)) == binding.SCD_ERR_UNSUPPORTED


def test_exact_plan_validation(lib):
    """Exact-length plans reject bad arguments before touching a device."""
    h = ctypes.c_void_p()
    arr = (ctypes.c_int64 * 2)(5000, 6000)
    assert lib.scd_batch_plan_create_exact(1, 0, arr, 32, 1, 0, ctypes.byref(h)) == binding.SCD_ERR_ARG
    assert lib.scd_batch_plan_create_exact(2, 2, arr, 32, 1, 0, ctypes.byref(h)) == binding.SCD_ERR_ARG
    assert lib.scd_batch_plan_create_exact(1, 2, arr, 24, 1, 0, ctypes.byref(h)) == binding.SCD_ERR_UNSUPPORTED
    assert lib.scd_batch_plan_create_exact(0, 2, arr, 32, 0, 0, ctypes.byref(h)) == binding.SCD_ERR_ARG
    assert lib.scd_batch_plan_create_exact(1, 2, arr, 32, 1, 7, ctypes.byref(h)) == binding.SCD_ERR_UNSUPPORTED
    assert lib.scd_batch_plan_create_exact(1, 2, None, 32, 1, 0, ctypes.byref(h)) == binding.SCD_ERR_ARG


def test_noalloc_argument_validation(lib):
    """scd_fam_noalloc applies scd_fam's checks, then its own limits; every rejection comes
    before any CUDA call and leaves a message in scd_last_error()."""
    assert lib.scd_fam_noalloc(FAKE, 279, 32, 8, 32, None, FAKE, None) == binding.SCD_ERR_ARG
    assert lib.scd_fam_noalloc(FAKE, 280, 24, 8, 32, None, FAKE, None) == binding.SCD_ERR_UNSUPPORTED
    assert lib.scd_fam_noalloc(FAKE, 1 << 20, 32, 8, 100, None, FAKE, None) == binding.SCD_ERR_UNSUPPORTED
    assert b"power of two" in lib.scd_last_error()
    assert lib.scd_fam_noalloc(FAKE, 1 << 20, 256, 64, 2048, None, FAKE, None) == binding.SCD_ERR_UNSUPPORTED
    assert b"scratch limit" in lib.scd_last_error()
    assert lib.scd_fam_noalloc(FAKE, 1 << 20, 32, 8, 1 << 16, None, FAKE, None) == binding.SCD_ERR_UNSUPPORTED
    # the check that scd_fam has and the first version of this entry point lacked
    assert lib.scd_fam_noalloc(FAKE, 1 << 32, 16, 1 << 20, 4096, None, FAKE, None) == binding.SCD_ERR_UNSUPPORTED


def test_host_buffer_calls_validation(lib):
    """The host-buffer batch calls and the page-locked allocator reject bad arguments before
    any CUDA call: no plan, NULL device or host pointers, misaligned device pointers, a zero
    size; freeing NULL is a no-op."""
    p = ctypes.c_void_p
    assert lib.scd_batch_run_host(None, None, FAKE, None, FAKE, FAKE, FAKE, None) == binding.SCD_ERR_ARG
    assert lib.scd_batch_host_wait(None) == binding.SCD_ERR_ARG
    ptr = p()
    assert lib.scd_host_alloc(0, ctypes.byref(ptr)) == binding.SCD_ERR_ARG
    assert lib.scd_host_alloc(16, None) == binding.SCD_ERR_ARG
    assert lib.scd_host_free(None) == binding.SCD_OK
