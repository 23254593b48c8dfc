"""Host-side bookkeeping of bench.py: the algorithmic HBM bytes per site the
orbital-storage roofline counts for each kernel choice, the kernel that
lbks_relax_step_psi runs for each forced mode, and the ncu traffic record of
the stream-collide kernel matching its current source."""
import json
import os

import bench


class _Shape:
    """The two fields the byte model reads: orbital count and grid."""

    def __init__(self, n_orb, nx=128):
        self.n_orb, self.n = n_orb, (nx, 128, 128)


def _w(n_orb, nx=128):
    return _Shape(n_orb, nx)


def test_orbital_storage_bytes_per_site():
    # up to eight orbitals: psi in and out, Vc (FP64) once
    name, b = bench.psi_step_kernels(_w(5), 4, 0)
    assert name == "k_relax_psi_tile" and b == 4 * 10 + 8
    assert bench.psi_step_kernels(_w(5), 8, 2) == ("k_relax_psi_tma", 8 * 10 + 8)
    # forty orbitals, W-field path: + the overlap's read of psi', the W field's read of psi,
    # its write of u (39) and the stencil's read of u (39)
    name, b = bench.psi_step_kernels(_w(40), 4, 0)
    assert b == 4 * (80 + 4 * 40 - 2) + 8
    assert name.startswith("k_w_field_wide + k_relax_psi_wide_tile + k_gram_tc")
    # forty orbitals through the TMA step: psi in and out, the overlap's read of psi'
    name, b = bench.psi_step_kernels(_w(40), 4, 2)
    assert b == 4 * 120 + 8 and name.startswith("k_relax_psi_tma + k_gram_tc")


def test_kernel_for_each_forced_mode():
    w, ragged = _w(5, 128), _w(5, 130)  # 128: whole 16-byte rows in FP32; 130: not (FP64: yes)
    assert [bench.psi_kernel_index(w, 4, m) for m in range(5)] == [2, 0, 1, 2, 3]
    assert [bench.psi_kernel_index(ragged, 4, m) for m in range(5)] == [0, 0, 1, 0, 3]
    assert bench.psi_kernel_index(_w(40, 128), 4, 4) == 0  # more than eight orbitals: tiled
    assert bench.psi_kernel_index(ragged, 8, 0) == 2


def test_traffic_record_matches_the_kernel_source():
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "stream_collide_ch4_128_fp32.json")))
    assert rec["kernel_src_sha256"] == bench.kernel_source_sha()
    assert bench.recorded_traffic() == float(rec["dram_bytes_per_launch"])


def test_nearest_rank_percentiles():
    v = sorted(float(i) for i in range(1, 201))  # 1 .. 200
    assert bench.percentile(v, 0.5) == 100.0
    assert bench.percentile(v, 0.99) == 198.0  # the 198th of 200: not the maximum
    assert bench.percentile(v, 1.0) == 200.0
    s = bench.latency_summary(v)
    assert s["n"] == 200 and s["max"] == 200.0 and s["p90"] == 180.0
    assert bench.percentile([3.0], 0.99) == 3.0


def test_concurrent_oracle_rate():
    """Whole-host rate: every process's timed updates over the slowest
    process's timed seconds (warm-up steps skipped)."""
    a = {"times": [9.0, 1.0, 1.0], "updates_per_step": 1e9}
    b = {"times": [9.0, 2.0, 2.0], "updates_per_step": 1e9}
    value, steps, t = bench.oracle_rate([a, b], skip=1)
    assert steps == 4 and t == 4.0 and value == 1.0  # 4e9 updates / 4 s = 1 GLUPS


def test_wide_traffic_record_matches_the_kernel_sources():
    rec = json.load(open(bench.WIDE_TRAFFIC_FILE))
    assert rec["sources_sha256"] == bench.wide_sources_sha()
    assert bench.recorded_wide_traffic(1000) == 1000 * float(rec["dram_bytes_per_orbital_site"])


def test_wide_pair_traffic_record_matches_the_kernel_sources():
    rec = json.load(open(bench.WIDE_PAIR_TRAFFIC_FILE))
    assert rec["variant"] == "pairs"
    assert rec["sources_sha256"] == bench.wide_sources_sha(1)
    assert bench.recorded_wide_traffic(1000, 1) == 1000 * float(rec["dram_bytes_per_orbital_site"])
    assert bench.recorded_wide_traffic(1000, 2) is None  # no record for the prefetch variant
