"""bench.py's CPU baseline legs on a small workload, on CPU: the oracle
sample grows its window until the run is long enough, reuses a given
window size unchanged, and the single-thread leg leaves the oracle's thread
count as it found it."""
import bench
import oracle
import workloads


def test_sample_search_and_fixed_window():
    W = workloads.tangled(24, seed=2)
    r, el, nz = bench.cpu_oracle_sample(W, target_seconds=0.0)
    assert nz == 4 and r["value"] > 0 and r["kind"] == "oracle"
    assert "4x24x24 window" in r["sample"]
    r2, el2, nz2 = bench.cpu_oracle_sample(W, target_seconds=1e9, size=8)
    assert nz2 == 8 and "8x24x24 window" in r2["sample"]
    # a window larger than the grid is clamped to it
    r3, _, nz3 = bench.cpu_oracle_sample(W, target_seconds=1e9, size=100)
    assert nz3 == 24


def test_single_thread_leg_restores_threads():
    W = workloads.tangled(24, seed=2)
    before = oracle.set_threads(0)
    cpu = bench.cpu_baseline_all_and_one(W)
    assert oracle.set_threads(0) == before
    assert cpu["cores"] == before
    assert cpu["single_thread"]["value"] > 0
    assert "logical CPUs" in cpu["host"]
