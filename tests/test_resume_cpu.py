"""Resumable rate sets (paper_2104_04895_gb300.resume), host logic on the CPU.

The library's rate call is replaced by a stand-in with the same interface that evaluates the selected modes with
the oracle (each mode's rate is its own sum, Eq. tao0), so the slicing, the checkpoint files, the manifest check
and the resume can be tested without a GPU.  The GPU side of a slice is fp_rates4 with a mode mask, which the
GPU parity tests cover.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2104_04895_gb300 import resume, synth
from paper_2104_04895_gb300.sharding import pair_units

from conftest import oracle_modes


class OracleCtx:
    """Stand-in for binding.Context: rates4 with a mode mask, computed by the oracle; fails on call `fail_on`."""

    def __init__(self, cr, fail_on=None):
        self.cr, self.grid, self.N, self.nb = cr, tuple(cr.grid), cr.nq, cr.nb
        self.w, self.e, self.v = oracle_modes(cr)
        self.calls, self.fail_on = 0, fail_on

    def rates4(self, temps, scalebroad, mode_mask=None, **opts):
        self.calls += 1
        if self.fail_on is not None and self.calls == self.fail_on:
            raise RuntimeError("injected failure of a slice")
        sel = np.nonzero(mode_mask)[0]
        r, acc = oracle.rates4(self.cr, self.w, self.e, self.v, temps=temps, scalebroad=scalebroad, sel=sel)
        out = np.zeros((len(temps), self.N * self.nb))
        out[:, sel] = r
        return out.reshape(len(temps), self.N, self.nb), {"accepted": list(acc), "candidates": 3.0 * len(sel) *
                                                          self.N ** 2 * self.nb ** 3, "ms": 1.0}


@pytest.fixture(scope="module")
def case():
    cr = synth.diamond_si((3, 2, 2))
    w, e, v = oracle_modes(cr)
    temps = [300.0, 600.0]
    full, acc = oracle.rates4(cr, w, e, v, temps=temps)
    return cr, temps, full.reshape(len(temps), cr.nq, cr.nb), acc


def test_slices_cover_the_grid_in_whole_pairs():
    grid = (4, 3, 2)
    plan = resume.plan_slices(grid, 5)
    qs = sorted(q for s in plan for q in s)
    assert qs == list(range(24))
    owner = {q: k for k, s in enumerate(plan) for q in s}
    for u in pair_units(grid):
        assert len({owner[q] for q in u}) == 1
    sizes = [len([u for u in pair_units(grid) if owner[u[0]] == k]) for k in range(5)]
    assert max(sizes) - min(sizes) <= 1


def test_sliced_run_equals_the_whole_grid(tmp_path, case):
    cr, temps, full, acc = case
    ctx = OracleCtx(cr)
    r, st = resume.rates4_resumable(ctx, temps, cr.scalebroad, str(tmp_path / "ck"), 4)
    assert np.array_equal(r, full)
    assert np.array_equal(np.array(st["accepted"]), acc)
    assert st["slices_computed"] == 4 and st["slices_loaded"] == 0 and ctx.calls == 4


def test_resume_after_a_failed_slice(tmp_path, case):
    cr, temps, full, acc = case
    ck = str(tmp_path / "ck")
    with pytest.raises(RuntimeError, match="injected"):
        resume.rates4_resumable(OracleCtx(cr, fail_on=3), temps, cr.scalebroad, ck, 5)
    done = sorted(f for f in os.listdir(ck) if f.startswith("slice_"))
    assert done == ["slice_0000.npz", "slice_0001.npz"]
    # a temporary file left by an interrupted write does not count as a finished slice
    with open(os.path.join(ck, "slice_0002.npz.tmp123.npz"), "wb") as f:
        f.write(b"partial")
    ctx = OracleCtx(cr)
    r, st = resume.rates4_resumable(ctx, temps, cr.scalebroad, ck, 5)
    assert ctx.calls == 3 and st["slices_loaded"] == 2 and st["slices_computed"] == 3
    assert np.array_equal(r, full)
    assert np.array_equal(np.array(st["accepted"]), acc)
    # a third run only loads
    ctx = OracleCtx(cr)
    r2, st2 = resume.rates4_resumable(ctx, temps, cr.scalebroad, ck, 5)
    assert ctx.calls == 0 and st2["slices_loaded"] == 5 and np.array_equal(r2, r)


def test_checkpoints_of_another_run_are_refused(tmp_path, case):
    cr, temps, _, _ = case
    ck = str(tmp_path / "ck")
    resume.rates4_resumable(OracleCtx(cr), temps, cr.scalebroad, ck, 2)
    for kw in (dict(temps=[300.0]), dict(scalebroad=0.5), dict(n_slices=3)):
        args = dict(temps=temps, scalebroad=cr.scalebroad, n_slices=2)
        args.update(kw)
        with pytest.raises(ValueError, match="another run"):
            resume.rates4_resumable(OracleCtx(cr), args["temps"], args["scalebroad"], ck, args["n_slices"])
    with pytest.raises(ValueError, match="another run"):
        resume.rates4_resumable(OracleCtx(cr), temps, cr.scalebroad, ck, 2, window=3.0)
    with pytest.raises(ValueError, match="per slice"):
        resume.rates4_resumable(OracleCtx(cr), temps, cr.scalebroad, str(tmp_path / "other"), 2, q_begin=1)


def test_costs_shape_the_plan():
    grid = (4, 4, 2)
    costs = np.ones(32)
    costs[0] = 100.0
    plan = resume.plan_slices(grid, 3, costs)
    heavy = [k for k, s in enumerate(plan) if 0 in s][0]
    assert len(plan[heavy]) < min(len(s) for k, s in enumerate(plan) if k != heavy)


def test_command_line_resumes_from_its_checkpoints(tmp_path, monkeypatch, case):
    """`python -m paper_2104_04895_gb300 rta --checkpoint`: the command-line glue around the resumable rates, with
    the stand-in context in place of the library's (the command line itself is run on the GPU elsewhere)."""
    from paper_2104_04895_gb300 import __main__ as cli, binding

    cr, temps, full, acc = case
    made = []

    class CliCtx(OracleCtx):
        def __enter__(self):
            return self

        def __exit__(self, *exc):
            return False

        def modes(self):
            return self.w, self.e, self.v

    def from_crystal(crystal, device=0):
        made.append(CliCtx(cr))
        return made[-1]

    monkeypatch.setattr(binding.Context, "from_crystal", staticmethod(from_crystal))
    args = ["rta", "--workload", "2", "--grid", *map(str, cr.grid), "--temps", *map(str, temps), "--no-nu-split",
            "--out", str(tmp_path / "run"), "--checkpoint", str(tmp_path / "ck"), "--slices", "3"]
    assert cli.main(args) == 0
    assert made[-1].calls == 3
    assert cli.main(args) == 0
    assert made[-1].calls == 0
    rows = np.loadtxt(os.path.join(tmp_path, "run", "T300K", "BTE.w_4ph"))
    np.testing.assert_array_equal(rows[:, -1], full[0].reshape(-1))
