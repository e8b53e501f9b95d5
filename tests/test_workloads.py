"""The seeded input generators: SplitMix64 against the known-answer outputs of its reference
implementation, and the recipe of the 256-instance batched workload (runs on CPU)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1812_11626_gb300 import workloads as W  # noqa: E402


def test_splitmix64_known_answers():
    """First outputs of the reference splitmix64 (Vigna's constants) seeded with 1234567."""
    g = W.SplitMix64(1234567)
    assert [g.next_u64() for _ in range(5)] == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                                                4593380528125082431, 16408922859458223821]


def test_uniform_is_the_top_53_bits():
    g, h = W.SplitMix64(1812), W.SplitMix64(1812)
    for _ in range(1000):
        u = g.uniform()
        assert 0.0 <= u < 1.0
        assert u == (h.next_u64() >> 11) / 2.0 ** 53


def test_batch_instances_recipe():
    """256 instances, N uniform over {50, 100, 200}, A in [0.5, 3), gamma = 10^U[-2, 0); the same
    draws on every call; the group sizes the batched bench reports."""
    b = W.batch_instances(256, 1812)
    assert b == W.batch_instances(256, 1812) and len(b) == 256
    assert all(x["N"] in (50, 100, 200) and 0.5 <= x["A"] < 3.0 and 0.01 <= x["gamma"] < 1.0 for x in b)
    counts = {n: sum(x["N"] == n for x in b) for n in (50, 100, 200)}
    assert counts == {50: 83, 100: 80, 200: 93}
    assert W.batch_instances(256, 1813) != b
