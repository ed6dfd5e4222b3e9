"""The error columns the precision sweep reports beside each format follow Table 2
of the paper (zfp's modes on C_d): bits per value, rate = 32 / bits per value,
RMSE, NRMSE = RMSE / range, the largest pointwise error and PSNR = 20 log10(range /
(2 RMSE)).  The definitions are pinned by the rows the paper prints
(tests/golden/table2_zfp_rows.txt) and by closed forms."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

ROWS = os.path.join(os.path.dirname(__file__), "golden", "table2_zfp_rows.txt")


def _rows():
    out = []
    for line in open(ROWS):
        if line.startswith("#") or not line.strip():
            continue
        mode, axis, *vals = [t.strip() for t in line.split("|")]
        out.append((mode, axis, *[float(v) for v in vals]))
    return out


@pytest.mark.parametrize("row", _rows(), ids=lambda r: f"{r[0]}-{r[1]}")
def test_psnr_and_rate_reproduce_the_printed_rows(row):
    mode, axis, bpv, rate, rmse, nrmse, maxerr, psnr = row
    # the printed NRMSE has three significant digits (at most 0.21 % off: 0.02 dB), PSNR two decimals
    assert abs(bench.psnr_db(nrmse) - psnr) <= 0.035
    # rate printed to two decimals
    assert abs(32.0 / bpv - rate) <= 0.006
    # the largest pointwise error bounds the RMSE
    assert rmse <= maxerr


def test_the_range_is_the_axis_matrix_s_in_every_mode():
    spans = {}
    for mode, axis, bpv, rate, rmse, nrmse, maxerr, psnr in _rows():
        spans.setdefault(axis, []).append(rmse / nrmse)
    for axis, s in spans.items():
        assert max(s) / min(s) < 1.01, axis  # NRMSE rounding only


def test_table2_metrics_closed_forms():
    # A spans [-1, 3]; every entry off by +-d: RMSE = largest error = d, NRMSE = d / 4
    A = np.linspace(-1.0, 3.0, 64 * 50).reshape(64, 50)
    d = 2.0 ** -20
    signs = np.where(np.arange(A.size).reshape(A.shape) % 2 == 0, 1.0, -1.0)
    m = bench.table2_metrics(A, A + d * signs, stored_bytes=A.size, values=A.size)
    assert m["rmse"] == pytest.approx(d, rel=1e-12)
    assert m["max_pointwise_error"] == pytest.approx(d, rel=1e-12)
    assert m["nrmse"] == pytest.approx(d / 4.0, rel=1e-12)
    assert m["psnr_db"] == round(20.0 * math.log10(4.0 / (2.0 * d)), 2)
    assert m["bits_per_value"] == 8.0 and m["rate"] == 4.0  # one byte per value: Table 2's fixed rate 8
    # one entry off by e: RMSE = e / sqrt(n)
    B = A.copy()
    B[3, 7] += 0.5
    m = bench.table2_metrics(A, B, stored_bytes=A.size * 2, values=A.size)
    assert m["rmse"] == pytest.approx(0.5 / math.sqrt(A.size), rel=1e-12)
    assert m["max_pointwise_error"] == 0.5 and m["bits_per_value"] == 16.0 and m["rate"] == 2.0
    assert bench.table2_metrics(A, A, 1, 1)["psnr_db"] is None  # lossless: no finite PSNR
    assert bench.psnr_db(0.0) == float("inf")
