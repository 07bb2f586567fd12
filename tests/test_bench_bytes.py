"""The byte counts bench.py divides by the measured launch times (the roofline's
numerators), checked against values fixed outside bench.py:

* the compulsory bytes of a staggered (E, H) node pair for the headline
  workload (n = 30, N_h = 57): 4 (n + N_h) bytes of int32 indices and
  s (2 n + N_h) bytes of weights in each pass, 5 field reals in the H pass
  (Ez gathered once, H read and written) and 4 in the E pass; 1668 B in FP32
  and 2640 B in FP64;
* the 16-bit index format: 2 bytes per entry plus the two 4-byte bases a
  32-node slice carries per stream (0.5 B per node for both streams), 4
  bytes per entry in slices that keep 32-bit entries;
* the collocated 2D step of the differentiation workload (n = 20, N_h = 31),
  each field read once and written once: 4 (20 + 31) = 204 B of indices,
  4 (2 * 20 + 31) + 4 * 2 * 20 = 444 B of weights and 10 field reals (40 B):
  688 B in FP32;
* the flops of one local weight system (the weight solve's roofline): the
  elimination of a K x (K + r) augmented matrix sums 2 j (j + r) over
  j < K, i.e. 2 [(K - 1) K (2K - 1) / 6 + r (K - 1) K / 2], plus r K^2 for
  the back substitutions.
"""
import pytest

import bench


def test_staggered_pair_bytes_fp32_and_fp64():
    assert sum(bench.algorithmic_bytes(30, 57, 4)) == 1668
    assert sum(bench.algorithmic_bytes(30, 57, 8)) == 2640
    h, e = bench.algorithmic_bytes(30, 57, 4)
    assert (h, e) == (836, 832)


def test_16_bit_format_bytes():
    sl = 31250  # 1M nodes in 32-node slices
    h, e = bench.format_bytes(30, 57, 4, {"h": (sl, 0, 0), "e": (sl, 0, 0)})
    assert h == pytest.approx(2 * 87 + 0.5 + 4 * 117 + 5 * 4)
    assert e == pytest.approx(2 * 87 + 0.5 + 4 * 117 + 4 * 4)
    # slices that keep 32-bit entries cost 2 more bytes per entry of that stream
    h1, _ = bench.format_bytes(30, 57, 4, {"h": (sl, sl, 0), "e": (sl, 0, 0)})
    assert h1 - h == pytest.approx(2 * 30)
    h2, _ = bench.format_bytes(30, 57, 4, {"h": (sl, sl, sl), "e": (sl, 0, 0)})
    assert h2 == pytest.approx(bench.algorithmic_bytes(30, 57, 4)[0] + 0.5)


def test_layouts_without_16_bit_streams_count_32_bit_indices():
    assert bench.format_bytes(30, 57, 4, {"h": (0, 0, 0), "e": (0, 0, 0)}) == bench.algorithmic_bytes(30, 57, 4)


def test_collocated_step_bytes():
    assert sum(bench.colloc_bytes(20, 31, 4)) == 204 + 444 + 40 == 688
    assert bench.colloc_bytes(20, 31, 4) == (432, 256)
    assert sum(bench.colloc_bytes(20, 31, 8)) == 204 + 2 * 444 + 80


def test_weight_solve_flops_closed_form():
    for K, r in ((45, 2), (85, 1), (106, 1), (62, 3)):
        closed = 2 * ((K - 1) * K * (2 * K - 1) // 6 + r * (K - 1) * K // 2) + r * K * K
        assert bench.solve_flops(K, r) == closed
    assert bench.solve_flops(45, 2) == 66750
    assert bench.poly_count(4) == 15 and bench.poly_count(6) == 28 and bench.poly_count(3, 3) == 20
