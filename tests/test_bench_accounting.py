"""The benchmark's algorithmic-byte accounting (host logic, no GPU).

bench.py turns the library's per-pass trace into the roofline figure: per
pass 4 bytes a scanned arc (target id), a row of W bytes per gathered
successor, own row read and row written, 8 n bytes of offsets in pull passes
and n/4 bytes of changed-node bitmaps.  Pass 0 reads a two-byte c_0 record
per successor and run instead of a row where the library has the records,
and the roofline's dominant launch is a dense pass that gathers rows.
"""
import bench


def row(t, mode, scanned, gathered, own, writes, ms=1.0):
    return {"t": t, "mode": mode, "arcs_scanned": scanned, "arcs_gathered": gathered,
            "own_reads": own, "writes": writes, "union_ms": ms}


def test_row_pass_bytes():
    n, W = 1000, 64
    r = row(3, 2, scanned=5000, gathered=4000, own=900, writes=800)
    expected = 4 * 5000 + W * (4000 + 900 + 800) + 8 * n + n / 4
    assert bench.union_bytes(r, n, W) == expected
    assert bench.union_bytes(r, n, W, record_bytes=2) == expected   # t > 0: rows


def test_pass0_counts_records_not_rows():
    n, W, R = 1000, 64, 1
    r = row(0, 2, scanned=5000, gathered=5000, own=1000, writes=1000)
    with_rows = bench.union_bytes(r, n, W)
    with_records = bench.union_bytes(r, n, W, record_bytes=2 * R)
    assert with_records == 4 * 5000 + 2 * (5000 + 1000) + W * 1000 + 8 * n + n / 4
    assert with_rows - with_records == (W - 2 * R) * (5000 + 1000)


def test_scatter_and_systolic_passes_have_no_offsets_term():
    n, W = 1000, 64
    for mode in (1, 3):
        r = row(5, mode, scanned=10, gathered=10, own=10, writes=10)
        assert bench.union_bytes(r, n, W) == 4 * 10 + W * 30 + n / 4


def test_dense_row_passes_leave_out_pass0_with_records():
    n, W = 1000, 64
    rows = [row(0, 2, 100, 100, 10, 10, ms=1.0), row(1, 2, 100, 100, 10, 10, ms=2.0),
            row(2, 2, 100, 100, 10, 10, ms=3.0), row(3, 0, 100, 50, 10, 10, ms=4.0),
            row(4, 3, 5, 5, 5, 5, ms=5.0)]
    ms, nbytes, count = bench.dense_row_passes(rows, n, W, record_bytes=2)
    assert (ms, count) == (5.0, 2)
    assert nbytes == sum(bench.union_bytes(r, n, W, 2) for r in rows[1:3])
    ms, nbytes, count = bench.dense_row_passes(rows, n, W)          # rows everywhere
    assert (ms, count) == (6.0, 3)
