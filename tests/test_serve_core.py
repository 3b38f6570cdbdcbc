"""CPU tests of the serving scheduler (queue, admission by HBM budget,
batching, LRU embedding cache, failures, timeouts, release) with a fake
backend: tests/serve_core_check.cpp is compiled against the CUDA-free core
paper_1406_6072_gb300/csrc/cf_serve_core.h and its JSON output checked."""
import json
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def scenarios():
    if not shutil.which("g++"):
        pytest.skip("g++ not available")
    d = tempfile.mkdtemp()
    exe = os.path.join(d, "serve_core_check")
    subprocess.run(["g++", "-std=c++17", "-O2", "-pthread", "-I", os.path.join(ROOT, "include"),
                    os.path.join(HERE, "serve_core_check.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120, check=True).stdout
    return {d["scenario"]: d for d in (json.loads(line) for line in out.splitlines() if line.strip())}


def test_mixed_requests_all_complete_with_batching(scenarios):
    s = scenarios["mixed"]
    assert s["ok"] == 60 and s["completed"] == 60
    assert s["batched_requests"] == 60 and s["batches"] < 60
    assert 0 < s["p50"] <= s["p99"] <= s["lat_max"] + 1e-9
    assert s["cache_misses"] == 3 * 4 - 0 or s["cache_misses"] >= 1
    assert s["allocs"] == s["frees"]
    assert s["embeds"] == s["cache_misses"]


def test_budget_bounds_device_memory(scenarios):
    s = scenarios["budget"]
    assert s["ok"] == 12
    assert s["peak"] <= s["budget"]
    assert s["batches"] == 12  # one request fits at a time


def test_request_larger_than_budget_is_rejected(scenarios):
    s = scenarios["reject"]
    assert s["big"] == 3  # CF_ERR_NOMEM
    assert s["small"] == 0


def test_not_psd_spectrum_fails_and_is_cached(scenarios):
    s = scenarios["notpsd"]
    assert s["a"] == 2 and s["b"] == 2  # CF_ERR_NOT_PSD
    assert s["b_hit"] == 1 and s["embeds"] == 1 and s["neg"] == 3


def test_queue_wait_and_release_semantics(scenarios):
    s = scenarios["queue"]
    assert s["sa"] == 0 and s["sb"] == 0 and s["sc"] == 0
    assert s["sd"] == 7          # CF_ERR_BUSY: queue capacity 2
    assert s["wait_short"] == 6  # CF_ERR_TIMEOUT
    assert s["release_early"] == 7
    assert s["wait_long"] == 0 and s["release"] == 0
    assert s["release_again"] == 8 and s["unknown"] == 8  # CF_ERR_NOT_FOUND


def test_stop_frees_everything(scenarios):
    s = scenarios["stop"]
    assert s["allocs"] == s["frees"]
    assert s["embeds"] == s["emb_frees"]


def test_lru_evicts_least_recently_used(scenarios):
    s = scenarios["lru"]
    assert s["evictions"] >= 1
    assert s["misses"] + s["hits"] == 6


def test_no_request_is_overtaken_by_more_than_a_batch(scenarios):
    s = scenarios["fifo"]
    assert s["started"] == 30
    assert s["max_delay"] <= 3  # max_batch_realizations


def test_slow_build_does_not_hold_up_ready_requests(scenarios):
    s = scenarios["overtake"]
    assert s["fast_ok"] == 10
    assert s["fast_max_ms"] < 150          # well under the 300 ms build
    assert s["slow"] == 0 and s["slow_status"] == 0
    assert s["slow_ms"] >= 300 and s["slow_hit"] == 0


def test_reserved_slot_serves_small_requests_beside_a_long_batch(scenarios):
    s = scenarios["reserved"]
    assert s["small_ok"] == 6
    assert s["small_max_ms"] < 200        # the long batch runs 800 ms
    assert s["big_ms"] >= 700
    assert s["big2_status"] == 0 and s["big2_queue_ms"] >= 500  # large requests keep to the general slot


def test_request_larger_than_a_batch_is_refused(scenarios):
    s = scenarios["oversize"]
    assert s["too_big"] == 1  # CF_ERR_ARG
    assert s["fits"] == 0 and s["status"] == 0
