"""Host logic of the benchmark that needs no GPU: the committed kernel profile
summary is keyed to the CUDA sources it was taken on, and the bench reads the
per-variant figures from it only for the profiled launch shapes."""
import bench


def test_profile_summary_matches_the_committed_sources():
    """The DRAM traffic and executed-instruction figures in the profile summary
    were taken on exactly these CUDA sources (a source change without a new
    capture would make the bench report figures of another kernel)."""
    kv, why = bench.profile_counters(32, 0)
    assert kv is not None, why
    assert kv["source_hash"] == bench.source_hash()


def test_profile_figures_per_variant_and_shape():
    k0, _ = bench.profile_counters(32, 0)
    k1, _ = bench.profile_counters(32, 1)
    assert int(k0["dram_bytes_per_launch"]) != int(k1["dram_bytes_per_launch"])
    assert 0.5 < float(k0["executed_per_algorithmic_flop"]) < 1.0
    assert 0.5 < float(k1["executed_per_algorithmic_flop"]) < 1.0
    assert "variant 0" in k0["small_case"] and "variant 1" in k1["small_case"]
    for tpc, var in ((64, 0), (32, 2), (128, 1)):
        kv, why = bench.profile_counters(tpc, var)
        assert kv is None and "launch shape" in why
