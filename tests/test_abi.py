"""The C-ABI library builds, loads and exports every entry point its header
declares; argument errors that are decided on the host come back as the
documented status codes.  No GPU needed: nothing here launches a kernel or
touches device memory."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2607_02630_gb300 import aesoffload as A
from paper_2607_02630_gb300 import build as B

HEADER = os.path.join(B.INCLUDE, "aesoffload.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return A.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    names = set(re.findall(r"\b((?:aes|offload)_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["aes_ctx_create", "aes_ctr", "aes_ctr_batch", "offload_submit", "offload_poll",
                 "offload_server_create", "offload_server_destroy", "aes_batch_plan_launch"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    for n in declared_functions():
        assert getattr(lib, n) is not None


def test_library_has_no_torch_or_python_dependency(lib):
    out = subprocess.run(["ldd", B.LIB], capture_output=True, text=True).stdout
    assert "torch" not in out and "python" not in out


def test_build_targets_sm_103a_only():
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_strings(lib):
    codes = [A.AES_OK, A.AES_PENDING, A.AES_EINVAL, A.AES_EKEYBITS, A.AES_EALIGN, A.AES_EOVERLAP,
             A.AES_EAGAIN, A.AES_ETIMEOUT, A.AES_ECUDA, A.AES_ESTOPPED, A.AES_ENOMEM, A.AES_ETOOBIG,
             A.AES_EPTR, A.AES_EDESC]
    names = [A.strerror(c) for c in codes]
    assert len(set(names)) == len(codes)
    assert all(n.startswith("AES_") for n in names)
    assert A.strerror(-999) == "unknown status"
    assert lib.aes_version() == 0x000100


def test_host_side_argument_errors(lib):
    h = ctypes.c_void_p()
    key = ctypes.create_string_buffer(32)
    iv = (ctypes.c_uint8 * 16)()
    assert lib.aes_ctx_create(None, key, 128) == A.AES_EINVAL
    assert lib.aes_ctx_create(ctypes.byref(h), None, 128) == A.AES_EINVAL
    for bits in (0, 64, 129, 512):
        assert lib.aes_ctx_create(ctypes.byref(h), key, bits) == A.AES_EKEYBITS
    assert h.value is None
    assert lib.aes_ctx_destroy(None) == A.AES_OK
    assert lib.aes_ctx_bits(None) == A.AES_EINVAL
    assert lib.aes_ctx_round_keys(None, key, 32) == A.AES_EINVAL
    assert lib.aes_ctr(None, iv, 16, 16, 16, None) == A.AES_EINVAL
    assert lib.aes_ctr_ex(None, iv, 16, 16, 16, None, None) == A.AES_EINVAL
    assert lib.aes_ctr_batch(None, -1, None) == A.AES_EINVAL
    assert lib.aes_ctr_batch(None, 5, None) == A.AES_EINVAL
    assert lib.aes_batch_plan_create(None, None, 1, None) == A.AES_EINVAL
    assert lib.aes_batch_plan_launch(None, None) == A.AES_EINVAL
    assert lib.aes_batch_plan_destroy(None) == A.AES_OK
    assert lib.aes_batch_plan_bytes(None) == A.AES_EINVAL
    t = ctypes.c_uint64()
    assert lib.offload_server_create(None, None) == A.AES_EINVAL
    assert lib.offload_submit(None, 0, iv, 16, 16, 16, ctypes.byref(t)) == A.AES_EINVAL
    assert lib.offload_poll(None, 1) == A.AES_EINVAL
    assert lib.offload_key_register(None, key, 128, None) == A.AES_EINVAL
    assert lib.offload_server_stats(None, None) == A.AES_EINVAL
    assert lib.offload_server_destroy(None) == A.AES_OK
    assert lib.aes_autotune_load(None) == A.AES_EINVAL
    assert lib.aes_tuned_shape(4096, 100, None) == A.AES_EINVAL
    assert lib.aes_batch_autotune(None, 0, None, None) == A.AES_EINVAL
    assert lib.aes_batch_autotune(None, 3, None, None) == A.AES_EINVAL
    assert lib.aes_batch_tuned_shape(None) == A.AES_EINVAL
    assert lib.aes_measure_peaks(None) == A.AES_EINVAL
    assert lib.aes_batch_tune_results(None, None, 4) == A.AES_EINVAL
    assert lib.aes_batch_tune_results(None, None, -1) == A.AES_EINVAL


def test_binding_refuses_to_run_without_library(tmp_path, monkeypatch):
    """No CPU fallback: a missing library is an error, not a silent path."""
    monkeypatch.setattr(B, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(A, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        A.lib()


# ctypes mirror (or numpy record) of each struct the header declares
MIRRORS = {
    "aes_launch_t": A.LaunchShape,
    "aes_desc_t": A.Desc,
    "aes_batch_opts_t": A.BatchOpts,
    "aes_peaks_t": A.Peaks,
    "offload_cfg_t": A.ServerCfg,
    "offload_stats_t": A.ServerStats,
    "aes_drive_result_t": A.DriveResult,
    "aes_drive_opts_t": A.DriveOpts,
    "cdet_run_cfg_t": A.CdetCfg,
    "cdet_run_result_t": A.CdetResult,
}
C_FIELD = {("aes_desc_t", "inp"): "in"}  # names that are Python keywords


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct the binding mirrors has the header's size and field
    offsets (the compiler's answer, from a C program built against the
    header), so a field added on one side only cannot shift the others."""
    drive = A.drive_dtype()
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "aesoffload.h"', "int main(void) {"]
    for cname, cls in MIRRORS.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            cf = C_FIELD.get((cname, f), f)
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {cf}));')
    lines.append('printf("aes_drive_req_t size %zu\\n", sizeof(aes_drive_req_t));')
    for f in drive.names:
        cf = "in" if f == "inp" else f
        lines.append(f'printf("aes_drive_req_t {f} %zu\\n", offsetof(aes_drive_req_t, {cf}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", B.INCLUDE, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {}
    for line in out.splitlines():
        t, f, v = line.split()
        got[(t, f)] = int(v)
    for cname, cls in MIRRORS.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)
    assert got[("aes_drive_req_t", "size")] == drive.itemsize
    for f in drive.names:
        assert got[("aes_drive_req_t", f)] == drive.fields[f][1], f


def test_short_keys_are_refused_before_the_library_reads_them():
    """The library reads bits / 8 key bytes; the binding refuses a shorter key
    instead of letting it read past the caller's buffer."""
    with pytest.raises(ValueError):
        A._keybuf(bytes(16), 256)
    with pytest.raises(ValueError):
        A._keybuf(bytes(23), 192)
    assert A._keybuf(bytes(32), 256) == bytes(32)
    assert A._keybuf(b"x", 64) == b"x"  # a key size the library rejects itself (AES_EKEYBITS)


def test_trace_build_builds_and_exports_its_reader():
    """The served path's trace build (-DSRV_TRACE) compiles, links, and
    exports offload_server_trace like the normal library."""
    path = B.build_trace()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert "offload_server_trace" in exported and "offload_submit" in exported


def test_iv_marshalling():
    """The initial counter block reaches the library as 16 bytes, from bytes,
    bytearray or a uint8 array, by pointer for the calls and as a uint8[16]
    for descriptors; any other length is refused before the call."""
    import numpy as np

    from paper_2607_02630_gb300 import aesoffload as A

    want = bytes(range(16))
    for iv in (want, bytearray(want), np.arange(16, dtype=np.uint8)):
        assert A._iv_bytes(iv) == want
        assert bytes(A._bytes16(iv)) == want
    for bad in (b"", bytes(15), bytes(17), np.zeros(8, dtype=np.uint16)[:7]):
        with pytest.raises(ValueError):
            A._iv_bytes(bad)
