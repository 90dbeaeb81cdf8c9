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
