"""The benchmark's DRAM traffic records (profiles/dram_traffic.txt), on CPU.

Each record holds one ncu capture's DRAM bytes for a kernel, keyed by the
hash of the kernel's source file.  bench.py reports the figure as a
roofline's `traffic` only while that source is unchanged, scaled per launch
or per block.  These tests check the records' format and that lookup rule;
they do not require the recorded hashes to match the current sources (a
kernel changed since its capture reports no traffic until it is captured
again).
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

RECORDS = os.path.join(ROOT, "profiles", "dram_traffic.txt")


def _records():
    with open(RECORDS) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_records_are_well_formed():
    recs = _records()
    assert recs
    names = [r[0] for r in recs]
    assert len(names) == len(set(names)), "one record per kernel"
    for r in recs:
        assert len(r) >= 6, r
        kernel, src, sha, nbytes, scale = r[:5]
        assert os.path.exists(os.path.join(ROOT, src)), src
        assert len(sha) == 12 and all(ch in "0123456789abcdef" for ch in sha), sha
        assert float(nbytes) > 0
        assert scale == "per_block" or float(scale) > 0
        with open(os.path.join(ROOT, src)) as f:
            assert kernel in f.read(), (kernel, src)     # the kernel lives in that file


def test_lookup_follows_the_source_hash(monkeypatch):
    recs = {r[0]: r for r in _records()}
    # every record as if its source were unchanged
    by_src = {r[1]: r[2] for r in recs.values()}
    monkeypatch.setattr(bench, "source_sha", lambda rel: by_src.get(rel))
    for kernel, r in recs.items():
        if r[4] == "per_block":
            assert bench.captured_traffic(kernel) is None          # needs the blocks per launch
            assert bench.captured_traffic(kernel, blocks_per_launch=4) == float(r[3]) * 4
        else:
            assert bench.captured_traffic(kernel) == float(r[3]) * float(r[4])
    # a changed source hides the record
    monkeypatch.setattr(bench, "source_sha", lambda rel: "000000000000")
    for kernel in recs:
        assert bench.captured_traffic(kernel, blocks_per_launch=4) is None
    assert bench.captured_traffic("no_such_kernel") is None


def test_operator_product_bytes_count_the_chunk_table():
    # blocks of 65, 64 and 1 rows: chunks of up to 64 rows -> 2 + 1 + 1 = 4
    ptr = [0, 65, 129, 130]
    n, c, nnz = 130, 8, 500
    want = n * c * 8 + nnz * 2 + (n + 1) * 4 + n * 4 + 4 * 32
    assert bench.spmm_algorithmic_bytes(n, c, nnz, ptr) == want
    # a 64^2 grid in four 32 x 32 tiles: 16 chunks per block
    from paper_1810_02719_gb300 import synth
    ptr, _ = synth.tile_partition(64, 32)
    assert bench.spmm_algorithmic_bytes(64 * 64, 1, 0, ptr) == \
        64 * 64 * 8 + (64 * 64 + 1) * 4 + 64 * 64 * 4 + 4 * 16 * 32
