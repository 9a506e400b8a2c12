"""The served kernel's request protocol, run by host threads on the CPU.

served_protocol.cuh holds the protocol (queue entries, dispatch into device
records, tile claims by either the global cursor or per-request claim words,
completion of a request's last tile) in code that compiles for the device
and, with GCC atomics, for the host.  served_protocol_sim.cpp runs it with
threads standing in for the resident CTAs (agent + worker each) against a
producer that submits and reaps requests as offload_submit / offload_poll
do, and checks that every tile is processed exactly once while its request
owns the slot and that every request completes once with its status.  The
settings mix slot reuse (down to one slot), more CTAs than cores, and idle
timeouts short enough to make CTAs exit and be relaunched under load."""
import os
import subprocess

import pytest

from paper_2607_02630_gb300 import build as B

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def sim(tmp_path_factory):
    nvcc = B._nvcc()
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    exe = str(tmp_path_factory.mktemp("sim") / "served_protocol_sim")
    # undefined behaviour aborts the run (and so fails the test)
    subprocess.run(["g++", "-O2", "-std=c++17", "-pthread", "-Wall", "-Wno-unknown-pragmas", "-fsanitize=undefined",
                    "-fno-sanitize-recover=undefined", "-I", B.INCLUDE,
                    "-I", B.CSRC, "-I", cuda_inc, os.path.join(HERE, "served_protocol_sim.cpp"), "-o", exe],
                   check=True)
    return exe


# ctas, slots, requests, tile_blocks (0 = per request), idle timeout us, seed
CASES = [
    (4, 32, 3000, 0, 2000, 7),
    (4, 32, 2000, 64, 2000, 8),
    (4, 32, 2000, 1024, 2000, 9),
    (2, 4, 3000, 0, 2000, 11),
    (16, 8, 3000, 64, 500, 12),
    (12, 64, 4000, 0, 300, 13),
    (3, 1, 1000, 0, 2000, 15),
]


@pytest.mark.parametrize("mode", [0, 1], ids=["global_cursor", "per_request"])
@pytest.mark.parametrize("case", CASES, ids=[f"c{c[0]}s{c[1]}t{c[3]}i{c[4]}" for c in CASES])
def test_every_tile_once_every_request_once(sim, mode, case):
    r = subprocess.run([sim, str(mode)] + [str(x) for x in case], capture_output=True, text=True, timeout=240)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr


@pytest.mark.parametrize("mode", [0, 1], ids=["global_cursor", "per_request"])
@pytest.mark.parametrize("case", [(4, 32, 3000, 0, 2000, 22), (8, 4, 2000, 64, 500, 24)], ids=["wide", "tight"])
def test_stop_flag_with_work_in_flight(sim, mode, case):
    """Every stand-in CTA exits once the stop flag is raised mid-run, with
    no tile processed twice."""
    r = subprocess.run([sim, str(mode)] + [str(x) for x in case] + ["1"], capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr


@pytest.mark.parametrize("mode", [0, 1], ids=["global_cursor", "per_request"])
def test_invalid_queue_entry_stops_with_error(sim, mode):
    """A queue entry naming a slot the host never issues stops the CTAs with
    status ERROR instead of leaving them waiting on it."""
    r = subprocess.run([sim, str(mode), "4", "32", "3000", "0", "2000", "23", "2"], capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr
    assert "status=" in r.stdout and int(r.stdout.split("status=")[1].split()[0]) & 4


# ctas, slots, requests, tile_blocks, idle us, seed, scenario, chaos period
CHAOS = [
    (8, 4, 1500, 0, 2000, 52, 0, 2),
    (4, 1, 600, 64, 2000, 61, 0, 3),
    (12, 16, 2000, 0, 500, 62, 0, 4),
    (4, 16, 1000, 0, 5000, 63, 1, 3),
]


@pytest.mark.parametrize("mode", [0, 1], ids=["global_cursor", "per_request"])
@pytest.mark.parametrize("case", CHAOS, ids=[f"c{c[0]}s{c[1]}sc{c[6]}ch{c[7]}" for c in CHAOS])
def test_under_schedule_perturbation(sim, mode, case):
    """The same checks with every protocol memory operation yielding the
    thread at random (1 in `chaos`), so the steps of different CTAs and the
    producer interleave far more finely."""
    r = subprocess.run([sim, str(mode)] + [str(x) for x in case], capture_output=True, text=True, timeout=240)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr


# ctas, slots, requests, tile_blocks, idle us, seed, scenario, chaos period, weak stores
WEAK = [
    (8, 8, 2000, 0, 2000, 81, 0, 0, 1),
    (4, 2, 1000, 64, 2000, 82, 0, 3, 1),
    (12, 32, 2000, 1024, 500, 83, 0, 0, 1),
    (4, 16, 1000, 0, 5000, 84, 1, 0, 1),
    (4, 16, 1000, 0, 5000, 85, 2, 0, 1),
]


@pytest.mark.parametrize("mode", [0, 1], ids=["global_cursor", "per_request"])
@pytest.mark.parametrize("case", WEAK, ids=[f"c{c[0]}s{c[1]}t{c[3]}sc{c[6]}ch{c[7]}" for c in WEAK])
def test_with_weak_store_visibility(sim, mode, case):
    """The same checks with stores that become visible late and out of order
    unless a fence orders them, as the device's relaxed stores may: every
    fence the protocol relies on is exercised (the per-request dispatch
    without its fence fails here)."""
    r = subprocess.run([sim, str(mode)] + [str(x) for x in case], capture_output=True, text=True, timeout=240)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr


@pytest.fixture(scope="module")
def sim_trace(tmp_path_factory):
    """The simulation with the protocol's trace stamps compiled in (-DSRV_TRACE)."""
    nvcc = B._nvcc()
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    exe = str(tmp_path_factory.mktemp("simtr") / "served_protocol_sim_trace")
    subprocess.run(["g++", "-O2", "-std=c++17", "-pthread", "-Wall", "-Wno-unknown-pragmas", "-DSRV_TRACE",
                    "-fsanitize=undefined", "-fno-sanitize-recover=undefined", "-I", B.INCLUDE, "-I", B.CSRC,
                    "-I", cuda_inc, os.path.join(HERE, "served_protocol_sim.cpp"), "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("mode", [0, 1], ids=["global_cursor", "per_request"])
@pytest.mark.parametrize("case", [(8, 8, 1500, 0, 2000, 5, 0, 2, 0), (4, 2, 1000, 64, 2000, 6, 0, 3, 1)],
                         ids=["plain", "weak"])
def test_trace_stamps_follow_the_protocol(sim_trace, mode, case):
    """Every request's trace stamps come in protocol order: dispatched,
    published, first claim, first pop, done (without tiles: dispatched,
    published, done)."""
    r = subprocess.run([sim_trace, str(mode)] + [str(x) for x in case], capture_output=True, text=True, timeout=240)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr


def soak_case(seed: int):
    """A configuration drawn from the seed: CTAs, slots, tile shape, idle
    timeout, scenario, perturbation and weak stores (reproducible)."""
    ctas = seed * 7 % 15 + 1
    slots = 1 << (seed % 7)
    tile_blocks = (0, 64, 256, 1024)[seed % 4]
    scenario = 1 if seed % 11 == 0 else (2 if seed % 13 == 0 else 0)
    idle_us = 400 if seed % 2 == 0 else 3000
    return [ctas, slots, 600, tile_blocks, idle_us, seed, scenario, seed % 5, (seed // 3) % 2]


@pytest.mark.parametrize("mode", [0, 1], ids=["global_cursor", "per_request"])
@pytest.mark.parametrize("seed", list(range(2000, 2024)))
def test_randomised_configurations(sim_trace, mode, seed):
    """Configurations drawn from seeds across every switch of the simulation
    (the trace build, so stamp order is checked too)."""
    r = subprocess.run([sim_trace, str(mode)] + [str(x) for x in soak_case(seed)], capture_output=True, text=True,
                       timeout=240)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr


def test_ring_placement_spreads_a_lease_over_partitions(tmp_path):
    """The agent's tile placement in its CTA ring (push_lease), on fixed
    cases: tiles of one lease go to workers on distinct SM partitions where a
    later waiting worker allows it, empty items stand in the skipped
    positions, unknown owners and room limits are respected, positions wrap
    around the ring."""
    nvcc = B._nvcc()
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    exe = str(tmp_path / "ring_placement_test")
    subprocess.run(["g++", "-O2", "-std=c++17", "-Wall", "-Wno-unknown-pragmas", "-fsanitize=undefined",
                    "-fno-sanitize-recover=undefined", "-I", B.INCLUDE, "-I", B.CSRC, "-I", cuda_inc,
                    os.path.join(HERE, "ring_placement_test.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr
