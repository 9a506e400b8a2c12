"""The page-protection conflict detector on its synthetic server (handlers
read a shared counter, park at an offload, write it back incremented), with a
host-timed offload, on the CPU (Sec. 5: unlocked shared aggregates lose
updates under overlap; the detector flags the conflicts and, enforcing,
re-runs conflicting handlers serialized)."""
import ctypes

import pytest

from paper_2607_02630_gb300 import aesoffload as A

N = 3000


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_02630_gb300 import build

    build.build()


def run(mode, counters=64, handlers=16, offload_ns=50_000, requests=N, emulate=True):
    return A.conflict_run(mode, handlers=handlers, requests=requests, counters=counters, offload_ns=offload_ns,
                          emulate_stores=emulate)


EMULATE = pytest.mark.parametrize("emulate", [True, False], ids=["emulated_stores", "unprotect"])


def test_unprotected_overlap_loses_updates():
    r = run(A.CDET_UNPROTECTED, counters=1)
    assert r["lost_updates"] > N // 2
    assert r["final_count"] + r["lost_updates"] == N
    assert r["conflicts"] == 0


def test_coarse_lock_loses_nothing():
    r = run(A.CDET_LOCK)
    assert r["lost_updates"] == 0 and r["final_count"] == N


@EMULATE
def test_detect_flags_every_lost_update(emulate):
    r = run(A.CDET_DETECT, emulate=emulate)
    assert r["lost_updates"] > 0
    assert r["conflicts"] >= r["lost_updates"]
    assert r["restarts"] == 0


@EMULATE
def test_enforce_loses_nothing(emulate):
    enf = run(A.CDET_ENFORCE, emulate=emulate)
    assert enf["lost_updates"] == 0 and enf["final_count"] == N
    assert enf["conflicts"] > 0 and enf["restarts"] == enf["conflicts"]


@EMULATE
def test_enforce_beats_the_coarse_lock(emulate):
    """The lock serializes every offload; enforcement serializes only the
    conflicting handlers (200 us offloads, so the detector's own fault costs,
    a few us each, stay small beside them)."""
    enf = run(A.CDET_ENFORCE, offload_ns=200_000, requests=1000, emulate=emulate)
    lock = run(A.CDET_LOCK, offload_ns=200_000, requests=1000)
    assert enf["lost_updates"] == 0
    assert enf["req_per_s"] > 1.5 * lock["req_per_s"]


def test_single_handler_never_conflicts():
    r = run(A.CDET_ENFORCE, counters=1, handlers=1, requests=300, offload_ns=10_000)
    assert r["lost_updates"] == 0 and r["conflicts"] == 0


@EMULATE
def test_false_sharing_is_conservative(emulate):
    """Counters sharing a page conflict at page granularity: more conflicts
    than with one counter per page, still no lost update when enforcing."""
    per_page = A.conflict_run(A.CDET_ENFORCE, handlers=16, requests=N, counters=64, counters_per_page=64,
                              emulate_stores=emulate)
    own_page = run(A.CDET_ENFORCE, emulate=emulate)
    assert per_page["lost_updates"] == 0
    assert per_page["conflicts"] > own_page["conflicts"]


def test_bad_arguments():
    with pytest.raises(A.AesError):
        A.conflict_run(A.CDET_LOCK, handlers=0)
    with pytest.raises(A.AesError):
        A.conflict_run(7)
    with pytest.raises(A.AesError):
        A.conflict_run(A.CDET_LOCK, counters_per_page=65)
    cfg = A.CdetCfg(16, 10, 64, 1, A.CDET_DETECT, 1000, None, 0, None, None, 0, 0, 2)  # no such store mode
    assert A.lib().cdet_run(ctypes.byref(cfg), ctypes.byref(A.CdetResult())) == A.AES_EINVAL


@EMULATE
@pytest.mark.parametrize("pattern", [A.CDET_PATTERN_READONLY, A.CDET_PATTERN_PER_CONN, A.CDET_PATTERN_LOCKED],
                         ids=["read_only", "per_connection", "lock_protected"])
def test_safe_patterns_raise_no_conflict(pattern, emulate):
    """The three shared-state patterns the paper finds safe under overlap
    (read-only, per-connection, lock-protected) lose nothing and make the
    detector report nothing; the hazardous one, on the same settings, does
    both."""
    r = A.conflict_run(A.CDET_DETECT, handlers=16, requests=2000, counters=64, pattern=pattern,
                       emulate_stores=emulate)
    assert r["conflicts"] == 0 and r["lost_updates"] == 0 and r["final_count"] == 2000, r
    hazard = A.conflict_run(A.CDET_DETECT, handlers=16, requests=2000, counters=64, emulate_stores=emulate)
    assert hazard["conflicts"] > 0 and hazard["lost_updates"] > 0


def test_per_connection_counters_sharing_a_page_are_flagged():
    """Per-connection counters packed onto one page lose no update but are
    flagged: the detector works at page granularity (conservative)."""
    r = A.conflict_run(A.CDET_DETECT, handlers=16, requests=2000, counters=64, counters_per_page=64,
                       pattern=A.CDET_PATTERN_PER_CONN)
    assert r["lost_updates"] == 0 and r["final_count"] == 2000
    assert r["conflicts"] > 0


def test_pattern_arguments():
    with pytest.raises(A.AesError):
        A.conflict_run(A.CDET_DETECT, pattern=4)
    with pytest.raises(A.AesError):  # per-connection needs a counter per handler
        A.conflict_run(A.CDET_DETECT, handlers=16, counters=8, pattern=A.CDET_PATTERN_PER_CONN)


def test_store_emulation_selftest():
    """Guarded stores of 8..64 bits at run-time offsets, performed by the
    fault handler, leave the region equal to a plain shadow copy; on x86-64
    and AArch64 the compiler's plain stores are all decoded."""
    import platform

    r = A.store_selftest(6000)
    assert r["emulated"] + r["fallbacks"] == 6000
    if platform.machine() in ("x86_64", "aarch64"):
        assert r["emulated"] == 6000 and r["fallbacks"] == 0, r


@pytest.mark.parametrize("mode", [A.CDET_DETECT, A.CDET_ENFORCE], ids=["detect", "enforce"])
def test_emulated_stores_keep_the_detectors_results(mode):
    """With store emulation the guarded pages never change protection and the
    detector reports what it reports without it: enforcement loses nothing,
    detection flags at least every lost update, safe patterns stay silent."""
    r = A.conflict_run(mode, handlers=16, requests=N, counters=64, emulate_stores=True)
    assert r["protect_calls"] == 0 and r["emulated_stores"] >= N, r
    if mode == A.CDET_ENFORCE:
        assert r["lost_updates"] == 0 and r["final_count"] == N and r["restarts"] == r["conflicts"] > 0
    else:
        assert r["lost_updates"] > 0 and r["conflicts"] >= r["lost_updates"]
    for pattern in (A.CDET_PATTERN_READONLY, A.CDET_PATTERN_PER_CONN, A.CDET_PATTERN_LOCKED):
        s = A.conflict_run(mode, handlers=16, requests=1000, counters=64, pattern=pattern, emulate_stores=True)
        assert s["conflicts"] == 0 and s["lost_updates"] == 0, (pattern, s)


def test_protection_changes_per_guarded_write():
    """One handler, no offload: each request's guarded write costs two
    protection changes (unprotect at the fault, protect again after the
    request), and none with store emulation."""
    n = 2000
    plain = A.conflict_run(A.CDET_DETECT, 1, n, 1, offload_ns=0, emulate_stores=False)
    emu = A.conflict_run(A.CDET_DETECT, 1, n, 1, offload_ns=0, emulate_stores=True)
    assert plain["final_count"] == n and emu["final_count"] == n
    assert plain["protect_calls"] == 2 * n and plain["emulated_stores"] == 0
    assert emu["protect_calls"] == 0 and emu["emulated_stores"] == n


@pytest.mark.parametrize("opt", ["-O0", "-O2"])
def test_detector_under_undefined_behaviour_sanitizer(tmp_path, opt):
    """conflict.cpp built on its own with -fsanitize=undefined (any finding
    aborts), run over every mode and pattern with and without store
    emulation, and its store self-test (the compiler's store forms differ
    between -O0 and -O2)."""
    import os
    import subprocess

    from paper_2607_02630_gb300 import build as B

    exe = str(tmp_path / "cdet_ubsan")
    here = os.path.dirname(os.path.abspath(__file__))
    subprocess.run(["g++", opt, "-g", "-std=c++17", "-fsanitize=undefined", "-fno-sanitize-recover=undefined",
                    "-I", B.INCLUDE, os.path.join(here, "conflict_ubsan_main.cpp"),
                    os.path.join(B.CSRC, "conflict.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "OK selftest rc=0" in r.stdout, r.stdout + r.stderr
