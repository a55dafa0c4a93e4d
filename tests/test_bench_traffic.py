"""The roofline's `traffic` comes from the ncu figures in profiles/
traffic.txt only while the pass kernels' sources are the ones they were
captured on (the sha stored beside each figure)."""
import bench


def test_committed_figures_match_the_sources():
    """profiles/traffic.txt carries figures for the current sources: the
    default keys and key+payload workloads at 2^26 have traffic and
    shared-memory wavefronts, within 15 % of the algorithmic bytes."""
    for key, algorithmic in (("onesweep_r8_keys_n67108864", 8 << 26), ("onesweep_r8_pairs_n67108864", 16 << 26)):
        t = bench.traffic_from_profiles(key)
        assert t is not None, f"{key}: no figure for sha {bench.pass_kernel_sha()}"
        assert 0.85 * algorithmic <= t <= 1.15 * algorithmic
        assert bench.traffic_from_profiles(key + "_smem_wavefronts") > 0


def test_a_changed_source_voids_the_figures(monkeypatch):
    monkeypatch.setattr(bench, "pass_kernel_sha", lambda: "0000000000000000")
    assert bench.traffic_from_profiles("onesweep_r8_keys_n67108864") is None
    assert bench.traffic_from_profiles("onesweep_r8_pairs_n67108864") is None
