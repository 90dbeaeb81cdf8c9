"""The SUPS metric reproduces the paper's printed numbers (Table III)."""
import os

from paper_1906_11925_gb300 import metrics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_table3_sups.txt")


def test_table3_sups():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 2
    for name, sites, seconds, steps, printed in rows:
        v = metrics.sups(int(sites), int(steps), float(seconds))
        assert int(v) == int(printed), (name, v, printed)


def test_bytes_per_site_update():
    assert metrics.bytes_per_site_update(15, "fp32") == 176
    assert metrics.bytes_per_site_update(15, "fp16") == 116
    assert metrics.bytes_per_site_update(19, "fp32") == 224
    assert metrics.bytes_per_site_update(19, "fp16") == 148
    assert metrics.bytes_per_site_update(19, "fp32", "aa") == 188
    assert metrics.bytes_per_site_update(19, "fp16", "aa") == 112
    assert metrics.bytes_per_site_update(19, "i16", "aa") == 112
    # fused step pairs: per step, half of (both passes' populations + one table read)
    assert metrics.bytes_per_site_update(19, "fp32", "aa_pairs") == 112
    assert metrics.bytes_per_site_update(19, "fp16", "aa_pairs") == 74


def test_profile_summaries_match_the_step_source():
    """The DRAM traffic the benchmark reports comes from the committed ncu
    summaries only while they name the hash of the current step-kernel
    source; a change to the step kernels without a new capture (or an
    explained hash update) shows here."""
    import bench

    for form in ("aa", "pull"):
        t = bench.recorded_traffic(bench.PROFILE_SUMMARY[("vessel_tree_large", form)])
        assert t is not None, form
        assert set(t) == {"traffic_bytes_per_launch_fp32", "traffic_bytes_per_launch_fp16"}
        # within a few percent of the algorithmic bytes of one bulk launch on
        # the at-scale tree (69.46M sites, about 69.34M without iolet links)
        bulk = 69_340_000
        alg = {"aa": (188, 112), "pull": (224, 148)}[form]
        assert 0.9 < t["traffic_bytes_per_launch_fp32"] / (alg[0] * bulk) < 1.1
        assert 0.9 < t["traffic_bytes_per_launch_fp16"] / (alg[1] * bulk) < 1.1
