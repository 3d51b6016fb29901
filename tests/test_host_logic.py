"""Host-side logic that needs no GPU: the storage-order helper, parameter
vector round trips, the ring-record binning, the desorption screening's
threshold rule (against a stand-in system object) and the benchmark's byte
accounting and peak lookup."""
import json
import os
import sys

import numpy as np
import pytest

from paper_1802_07871_gb300 import ctbop
from paper_1802_07871_gb300 import desorption as D
from paper_1802_07871_gb300 import rings as RG
from paper_1802_07871_gb300 import structures as st

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


# ---------------------------------------------------------------- storage order
def _grid(n):
    g = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    return g + 0.5


def test_morton_order_is_a_permutation_of_nested_cubes():
    """On a 4x4x4 grid with one atom per cell, every aligned run of 8 indices
    is a 2x2x2 cube and every run of 64 the whole grid (the defining
    property of a Z-order curve), whatever order the atoms come in."""
    x = _grid(4)
    rng = np.random.default_rng(1)
    x = x[rng.permutation(len(x))]
    o = ctbop.morton_order(x, np.full(3, 4.0), np.array([False] * 3), cell=1.0)
    assert sorted(o) == list(range(64))
    c = np.floor(x[o]).astype(int)
    for k in range(0, 64, 8):
        blk = c[k:k + 8]
        assert np.all(blk.max(0) - blk.min(0) == 1), blk
        assert np.all(blk.min(0) % 2 == 0)
        assert len({tuple(r) for r in blk}) == 8


def test_morton_order_wraps_periodic_axes():
    x = _grid(4)
    box, pbc = np.full(3, 4.0), np.array([True, True, False])
    shifted = x + np.array([4.0, -8.0, 0.0])          # whole periods on the periodic axes
    a = ctbop.morton_order(x, box, pbc, cell=1.0)
    b = ctbop.morton_order(shifted, box, pbc, cell=1.0)
    assert np.array_equal(a, b)


def test_morton_order_edge_cases():
    assert ctbop.morton_order(np.zeros((0, 3)), np.ones(3), np.zeros(3, bool)).shape == (0,)
    assert list(ctbop.morton_order(np.array([[1.0, 2.0, 3.0]]), np.full(3, 10.0), np.zeros(3, bool))) == [0]


# ---------------------------------------------------------------- parameters
def test_parameter_vector_round_trip():
    P = ctbop.params_struct(st.load_params("p1"))
    v = ctbop.params_vector(P)
    assert v.shape == (144,) and np.all(np.isfinite(v))
    assert bytes(ctbop.params_from_vector(v)) == bytes(P)
    with pytest.raises(ValueError):
        ctbop.params_from_vector(v[:-1])


# ---------------------------------------------------------------- ring records
def _records(rows):
    r = np.zeros(len(rows), dtype=ctbop.RING_DTYPE)
    for k, (rep, size, z, ang) in enumerate(rows):
        r[k]["replica"], r[k]["size"] = rep, size
        r[k]["centre"] = (0.0, 0.0, z)
        r[k]["orientation"] = ang
    return r


def test_ring_counts_and_orientation_histogram():
    rec = _records([(0, 6, 1.0, 5.0), (0, 6, 3.0, 59.9), (0, 5, 3.0, np.nan), (1, 7, 0.0, np.nan),
                    (1, 6, 4.0, 30.0), (2, 8, 0.0, np.nan), (2, 3, 0.0, np.nan)])
    c = RG.counts(rec, 3)
    assert c.shape == (3, 6)
    assert c[0].tolist() == [0, 0, 1, 2, 0, 0]
    assert c[1].tolist() == [0, 0, 0, 1, 1, 0]
    assert c[2].tolist() == [1, 0, 0, 0, 0, 1]
    h = RG.orientation_histogram(rec, bins=6)
    assert h.sum() == 3 and h[0] == 1 and h[3] == 1 and h[5] == 1
    assert RG.orientation_histogram(rec, bins=6, replica=0).sum() == 2
    assert RG.orientation_histogram(rec, bins=6, zmin=2.0).sum() == 2
    assert RG.counts(_records([]), 2).sum() == 0


# ---------------------------------------------------------------- desorption threshold
class _FakeSystem:
    """Stands in for ctbop.System: fixed coordination and removal energies."""

    def __init__(self, coord, energies):
        self.coord = np.asarray(coord, float)
        self.energies = dict(energies)

    def get(self, what):
        assert what == "coordination"
        return self.coord

    def removal_energies(self, cand, max_atoms=0):
        return np.array([self.energies[int(i)] for i in cand])


def test_screen_selects_mobile_undercoordinated_si_and_applies_thresholds():
    types = np.array([st.SI, st.SI, st.SI, st.C, st.SI, st.SI])
    frozen = np.array([False, False, False, False, True, False])
    coord = [3, 4, 2, 2, 3, 3]          # atom 1 is bulk, 3 is C, 4 is frozen
    energies = {0: 9.0, 2: 4.0, 5: 11.0}
    sysm = _FakeSystem(coord, energies)
    cand, dE, rm, thr = D.screen(sysm, types, frozen, threshold=6.5)
    assert cand.tolist() == [0, 2, 5] and dE.tolist() == [9.0, 4.0, 11.0]
    assert rm.tolist() == [2] and thr == 6.5
    # relative: the median of the 3-coordinated candidates (9, 11) less 3.5 eV
    cand, dE, rm, thr = D.screen(sysm, types, frozen, threshold="relative")
    assert thr == pytest.approx(10.0 - D.TERRACE_MARGIN)
    assert rm.tolist() == [2]
    with pytest.raises(ValueError):
        D.screen(sysm, types, frozen, threshold="median")
    # no candidate at all
    cand, dE, rm, thr = D.screen(_FakeSystem([4] * 6, {}), types, frozen, threshold="relative")
    assert len(cand) == len(dE) == len(rm) == 0 and thr == 0.0


# ---------------------------------------------------------------- benchmark accounting
@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    import bench as B
    return B


def test_matrix_pass_bytes(bench):
    # mixed: (int32 index + FP32 coefficient) per entry, 7 FP32 vectors + 8 B per atom
    assert bench.cg_matvec_bytes(10, 1000, 4) == 1000 * 8 + 10 * 36
    assert bench.cg_matvec_bytes(10, 1000, 8) == 1000 * 12 + 10 * 64
    assert bench.aggregate_value(1000, 10, 2, 500.0) == pytest.approx(1000 * 10 * 2 / 0.5)


def test_peak_comes_from_the_measured_file(bench):
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if not os.path.exists(path):      # written per machine; absent: the stated fallback
        assert bench.peaks() == (6800.0, "fallback")
        return
    with open(path) as f:
        hbm = float(json.load(f)["hbm_gbs"])
    assert bench.peaks() == (hbm, "measured")


# ---------------------------------------------------------------- caller buffers
def test_buffer_checks_reject_wrong_type_and_size():
    """A buffer the library would read or write past (too short, or of a
    narrower element type) is rejected on the host before any call."""
    chk = ctbop._check_buffer
    chk(np.zeros((4, 3)), np.float64, 12, "x")
    with pytest.raises(ValueError, match="12 elements"):
        chk(np.zeros((3, 3)), np.float64, 12, "x")
    with pytest.raises(TypeError, match="float64"):
        chk(np.zeros((4, 3), np.float32), np.float64, 12, "x")
    torch = pytest.importorskip("torch")
    chk(torch.zeros(4, 3, dtype=torch.float64), np.float64, 12, "x")
    chk(torch.zeros(5, dtype=torch.bool), np.uint8, 5, "frozen")
    chk(torch.zeros(5, dtype=torch.int32), np.int32, 5, "types")
    with pytest.raises(TypeError, match="float64"):
        chk(torch.zeros(4, 3, dtype=torch.float32), np.float64, 12, "x")
    with pytest.raises(TypeError, match="int32"):
        chk(torch.zeros(5, dtype=torch.int64), np.int32, 5, "types")
    with pytest.raises(ValueError, match="5 elements"):
        chk(torch.zeros(4, dtype=torch.uint8), np.uint8, 5, "frozen")
    with pytest.raises(TypeError):
        chk([0.0] * 12, np.float64, 12, "x")


def test_reference_arm_line(bench, monkeypatch, capsys):
    """`bench.py --impl reference` prints one JSON line in the benchmark's
    format, marked as the reference arm, its value the oracle's rate."""
    fake = {"value": 1234.5, "unit": bench.UNIT, "cores": 1, "kind": "oracle", "sample": "s"}
    monkeypatch.setattr(bench, "cpu_baseline", lambda **kw: dict(fake))
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "3", "--warmup", "1"])
    bench.main()
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["value"] == 1234.5 and line["unit"] == bench.UNIT and line["higher_is_better"] is True
    assert line["steps"] == 3 and line["warmup"] == 1 and line["n_gpus"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"] == {"value": 1234.5, "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == bench.WORKLOADS["1m"]


def test_cpu_baseline_times_the_oracle_on_a_bounded_sample(bench):
    cb = bench.cpu_baseline(steps=1, configs=False)
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] > 0
    assert "stepped 4H-SiC slab" in cb["sample"]


def test_cpu_baseline_all_cores_runs_one_process_per_core(bench):
    cb = bench.cpu_baseline_all_cores(steps=1)
    assert "unavailable" not in cb, cb
    assert cb["kind"] == "oracle" and cb["cores"] == (os.cpu_count() or 1) and cb["value"] > 0
    lo, hi = cb["per_process_min_max"]
    assert 0 < lo <= hi and cb["value"] >= cb["cores"] * lo * 0.999


def test_roofline_table_accounting(bench):
    """Per-phase roofline: per-step phases divide by the profiled steps, the
    CG phases by their launches; the binding bound is the largest fraction;
    the step fraction is the time-weighted mean over the covered phases."""
    n = 1000
    work = bench.phase_work(n, entries_all=230 * n, entries_mat=195 * n, n_cov_entries=5 * n,
                            bonds=4 * n, triplets=12 * n)
    assert work["bond"]["flops"] == 4 * n * 31 + 12 * n * 32
    assert work["cg_matvec"]["per"] == "launch"
    ph = {"bond": (2.0, 2), "cg_matvec": (3.0, 30), "lists": (1.0, 24)}
    peaks = {"fp32_tflops": 80.0, "mufu_ex2_tops": 5.0, "mufu_rsq_tops": 4.0}
    table, step = bench.roofline_table(ph, 2, work, peaks, 6000.0)
    assert set(table) == {"bond", "cg_matvec"}
    assert table["bond"]["ms_per_step"] == pytest.approx(1.0)
    assert table["cg_matvec"]["ms_per_launch"] == pytest.approx(0.1)
    hbm = work["cg_matvec"]["bytes"] / 1e-4 / 1e9 / 6000.0
    assert table["cg_matvec"]["bound"] == "hbm" and table["cg_matvec"]["frac"] == pytest.approx(hbm)
    for row in table.values():
        assert row["frac"] == pytest.approx(max(row["frac_by_bound"].values()), abs=1e-4)
    want = (2.0 * table["bond"]["frac"] + 3.0 * table["cg_matvec"]["frac"]) / 5.0
    assert step["frac"] == pytest.approx(want) and step["covered_share"] == pytest.approx(5.0 / 6.0)
