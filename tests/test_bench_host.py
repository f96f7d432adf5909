"""Host logic of bench.py (no GPU): the algorithmic byte count of a sweep against the printed
per-application totals for the 128^3 ILU(0) factors, the pencil grid of the partitioned schedule,
the empty-level chain of the latency floor, and the traffic figure read from a committed capture."""
import os
import sys

import numpy as np

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

N128 = 128 ** 3
NNZ_L_128 = 8_339_456  # ILU(0) of the 7-point matrix on 128^3, diagonal included (= nnz of U)


def test_sweep_bytes_match_the_printed_totals():
    # one L+U application: 250.9 MB with FP32 values, 317.6 MB with FP64, 1.26 GB for 16 columns
    lu = lambda sv, k: 2 * bench.sweep_bytes(NNZ_L_128, N128, k, sv)
    assert round(lu(4, 1) / 1e6, 1) == 250.9
    assert round(lu(8, 1) / 1e6, 1) == 317.6
    assert round(lu(4, 16) / 1e9, 2) == 1.26
    # the terms: values + indices, tail pointers, FP64 b read and x write, two index reads
    assert bench.sweep_bytes(10, 4, 1, 8) == 10 * 12 + 4 * 5 + 2 * 4 * 8 + 2 * 4 * 4


def test_sweep_grid_parts_fit():
    from paper_1606_00541_gb300 import synth
    for m, parts, crossings, threads in ((128, 256, 30, 512), (200, 152, 25, 1024)):
        nb = bench.sweep_grid(m)
        part, nparts = synth.grid_boxes(m, nb)
        assert nparts == parts and sum(k - 1 for k in nb) == crossings
        assert bench.part_threads(m) == threads
        # every part is an x-pencil whose FP32 solution fits the shared memory of its block: 227 KB
        # for one 1024-thread block an SM, half of the SM's 228 KB for two 512-thread blocks
        sizes = np.bincount(part, minlength=nparts)
        per_sm = 1 if threads == 1024 else 2
        assert sizes.min() > 0 and sizes.max() * 4 * per_sm <= 228 * 1024 - 1024 * per_sm
        assert nparts <= 152 * per_sm
        g = np.arange(m ** 3)
        y, z = (g // m) % m, g // (m * m)
        assert np.all(part == (y * nb[1]) // m + nb[1] * ((z * nb[2]) // m))


def test_chain_has_one_row_and_one_dependency_per_level():
    n = 64
    rp, ci, v = bench.chain_csr(n)
    assert oracle.check_triangular((rp, ci, v), 0) == 0
    lev, nlev = oracle.levels((rp, ci, v), 0)
    assert nlev == n and np.array_equal(lev, np.arange(n))
    assert np.array_equal(np.diff(rp), np.r_[1, np.full(n - 1, 2)])
    # well conditioned: for b = 1, x_i = 1 + x_{i-1} / 2, i.e. x_i = 2 - 2^-i
    x = oracle.lower_solve((rp, ci, v), np.ones(n))
    assert np.abs(x - (2.0 - 0.5 ** np.arange(n))).max() <= 4e-16


def test_recorded_traffic_follows_the_source_digest(monkeypatch, tmp_path):
    cap = tmp_path / "capture.md"
    cap.write_text("notes\n\ntraffic_bytes_per_launch: 107734400 source_digest: %s\n" % bench.sweep_source_digest())
    monkeypatch.setattr(bench, "SWEEP_PROFILES", {"part": str(cap), "global": str(tmp_path / "missing.md")})
    assert bench.recorded_traffic("part") == 107734400
    assert bench.recorded_traffic("global") is None  # no capture
    monkeypatch.setattr(bench, "sweep_source_digest", lambda: "0" * 16)
    assert bench.recorded_traffic("part") is None  # sources changed since the capture


def test_ras_pencil_grid_parts_fit():
    """The RAS form's subdomains, one partitioned part each, are all resident: the parts an SM
    needs fit its 64K registers at 60 a thread and its 228 KB of shared memory with FP64
    solutions (1 KB reserved a block); grids whose extended solution cannot fit are skipped."""
    from paper_1606_00541_gb300 import synth
    nb, threads = bench.ras_pencil_grid(128)
    A = synth.fv7_lognormal(128)
    part, ns = synth.grid_boxes(128, nb)
    ptr, _ = oracle.ras_extend(A, part, ns)
    per_sm = -(-ns // 152)
    assert per_sm * threads * 60 <= 65536
    assert per_sm * (int(np.diff(ptr).max()) * 8 + 1024) <= 228 * 1024
    assert bench.ras_pencil_grid(200) is None


def test_subdomain_parts_have_no_crossing_dependency():
    """Eq. 4: the RAS factors are block diagonal over the extended subdomains, so the part vector
    of bench.subdomain_parts (the subdomain of each extended row) puts both ends of every factor
    entry in the same part; the parts cover the extended rows in order."""
    from paper_1606_00541_gb300 import synth
    m = 12
    A = synth.fv7_lognormal(m, seed=4)
    part, ns = synth.grid_boxes(m, (2, 3, 3))
    R = oracle.ras_setup(A, part, ns)
    sp, nsp = bench.subdomain_parts(R["ext_ptr"])
    assert nsp == ns and len(sp) == R["ext_ptr"][-1]
    assert np.all(np.diff(sp) >= 0) and np.array_equal(np.bincount(sp, minlength=ns), np.diff(R["ext_ptr"]))
    for rp, ci, _ in (R["L"], R["U"]):
        rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
        assert np.array_equal(sp[rows], sp[ci])
