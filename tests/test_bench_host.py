"""Host-side arithmetic of the benchmark (CPU): the design bytes each kernel
kind moves per launch, the textbook bytes of a PCG step the roofline divides
by, the names of the PCG loops in the bench line, and the traffic lookup's
refusal of counters taken on other sources."""
import json

import bench

P = 640 * 480


def test_pcg_step_bytes_are_the_textbook_count():
    """(8 V + 2 + S) x 4 bytes per pixel: 360 B at V = 10 and S = 8 pair planes,
    110.6 MB at 640 x 480."""
    V, S = 10, 8
    assert 4 * (8 * V + 2 + S) == 360
    assert abs(4.0 * (8 * V + 2 + S) * P - 110.592e6) < 1.0


def test_design_bytes_of_the_two_kernel_loop():
    """k_apply reads z, the NC = 39 coefficient planes and (after step 1) p_old
    and q_old and writes p and q; k_update reads p, delta, z, q, M^-1 and writes
    delta and z (the last step: p, delta, X read, X written)."""
    K, M, ns, nt = 6, 20, 4, 1
    V, NC = K + 4, 10 + 3 * (K + 1) + 2 * ns
    assert NC == 39
    apply = bench.algorithmic_bytes("apply", K, P, M, ns, nt, True)
    assert abs(apply - 4.0 * P * ((M - 1) * (5 * V + NC) + (3 * V + NC)) / M) < 1e-6
    update = bench.algorithmic_bytes("update", K, P, M, ns, nt, True)
    assert abs(update - 4.0 * P * ((M - 1) * 7 * V + 4 * V) / M) < 1e-6
    # the persistent loop moves M operator and M vector phases per launch
    assert abs(bench.algorithmic_bytes("pcg", K, P, M, ns, nt, True) - M * (apply + update)) < 1e-3


def test_design_bytes_of_the_fused_step():
    """k_pcg_step reads z, M^-1 and the coefficients (+ mq_old, p_old, delta after
    step 1) and writes z, mq, p (+ delta): 9 V + NC planes per mid step, fewer
    than the two-kernel loop's 12 V + NC; its only vector-kernel launch is the
    last step's update (4 V planes)."""
    K, M, ns, nt = 6, 20, 4, 1
    V, NC = K + 4, 39
    fused = bench.algorithmic_bytes("apply", K, P, M, ns, nt, True, fused=True)
    assert abs(fused - 4.0 * P * ((M - 1) * (9 * V + NC) + (5 * V + NC)) / M) < 1e-6
    assert bench.algorithmic_bytes("update", K, P, M, ns, nt, True, fused=True) == 4.0 * P * 4 * V
    two_kernel_mid = 4.0 * P * (5 * V + NC + 7 * V)
    assert 4.0 * P * (9 * V + NC) < two_kernel_mid


class _Layout:
    def pcg_layout(self):
        return -1, (160, 13, 148)


def test_pcg_loop_names():
    assert "resident" in bench.pcg_loop_name(_Layout(), -1) and "160x13" in bench.pcg_loop_name(_Layout(), -1)
    assert bench.pcg_loop_name(_Layout(), 0) == "persistent PCG kernel"
    assert bench.pcg_loop_name(_Layout(), 17).startswith("128x17 operator tiles")
    assert "fused" in bench.pcg_loop_name(_Layout(), 17 | 256) and "128x17" in bench.pcg_loop_name(_Layout(), 273)
    assert bench.pcg_loop_name(_Layout(), 16).startswith("128x16 operator tiles")


def test_traffic_is_used_only_for_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    """profiles/traffic.json carries the hash of the kernel sources; a lookup
    against other sources returns None instead of stale counters."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"source_hash": bench.source_hash(), "kernels": {"pcg_step": {"dram_bytes_per_launch_full_size": 1.5e8}}}
    (prof / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_hash", lambda: rec["source_hash"])
    assert bench.ncu_traffic("pcg_step") == 1.5e8
    monkeypatch.setattr(bench, "source_hash", lambda: "0" * 16)
    assert bench.ncu_traffic("pcg_step") is None
