"""The onlyharmonic outputs (Sec. 2.1; BTE.Numprocess_4ph, BTE.P4, BTE.WP4 of Appendix A) against the oracle, the
FORCE_CONSTANTS_4TH round trip into the rate path, and the command-line tasks."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2104_04895_gb300 import bte, synth
from paper_2104_04895_gb300.binding import FP_PREC_DOUBLE_FLOAT, FP_PREC_MIXED

from conftest import oracle_modes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2104_04895_gb300 import binding
    binding.load()
    return binding


@pytest.mark.parametrize("maker", [lambda: synth.diamond_si((3, 3, 2)), lambda: synth.simple_cubic((4, 4, 4)),
                                   lambda: synth.licoo2((2, 2, 1))], ids=["diamond-3x3x2", "sc-4x4x4", "licoo2-2x2x1"])
def test_phase_space_matches_the_oracle(lib, maker):
    """Per-mode process counts exactly, P4 and WP4 to 1e-10 (FP64 and double-float paths, stride 1, time reversal
    folded); the mixed path keeps the counts and P4/WP4 within 2e-5."""
    cr = maker()
    w, e, v = oracle_modes(cr)
    temps = [300.0, 900.0]
    N, nb = cr.nq, cr.nb
    with lib.Context.from_crystal(cr) as ctx:
        ctx.set_modes(w, e, v)
        npr, p4, wp4 = ctx.phase_space4(temps, cr.scalebroad)
        nprm, p4m, wp4m = ctx.phase_space4(temps, cr.scalebroad, precision=FP_PREC_MIXED)
        nprd, p4d, wp4d = ctx.phase_space4(temps, cr.scalebroad, precision=FP_PREC_DOUBLE_FLOAT)
        with pytest.raises(lib.FourPhononError):
            ctx.phase_space4(temps, cr.scalebroad, stride=0)
    ref_p4, _ = oracle.rates4(cr, w, e, v, temps=temps[:1], unit_vertex=2)
    ref_wp4, acc = oracle.rates4(cr, w, e, v, temps=temps, unit_vertex=True)
    counts = np.array([oracle.rates4(cr, w, e, v, temps=temps[:1], sel=[m], unit_vertex=True)[1].sum()
                       for m in range(N * nb)])
    assert np.array_equal(npr, counts) and np.array_equal(nprm, counts) and np.array_equal(nprd, counts)
    assert npr.sum() == acc.sum() > 0
    ref_p4 = ref_p4[0] / N ** 2
    ref_wp4 = ref_wp4 / N ** 2
    pos = ref_p4 > 0
    assert np.all(p4[~pos] == 0.0) and np.all(wp4[:, ~pos] == 0.0)
    assert np.max(np.abs(p4[pos] - ref_p4[pos]) / ref_p4[pos]) <= 1e-10
    assert np.max(np.abs(wp4[:, pos] - ref_wp4[:, pos]) / ref_wp4[:, pos]) <= 1e-10
    assert np.max(np.abs(p4d[pos] - ref_p4[pos]) / ref_p4[pos]) <= 1e-10
    assert np.max(np.abs(wp4d[:, pos] - ref_wp4[:, pos]) / ref_wp4[:, pos]) <= 1e-10
    assert np.max(np.abs(p4m[pos] - ref_p4[pos]) / ref_p4[pos]) <= 2e-5
    assert np.max(np.abs(wp4m[:, pos] - ref_wp4[:, pos]) / ref_wp4[:, pos]) <= 2e-5


def test_phase_space_stride_scales_the_sample(lib):
    """stride s sums every s-th q' with all q'' and scales by s: its counts are estimates of the full counts."""
    cr = synth.diamond_si((4, 4, 4))
    with lib.Context.from_crystal(cr) as ctx:
        ctx.modes(copy=False)
        full, _, _ = ctx.phase_space4([300.0], cr.scalebroad)
        est, _, _ = ctx.phase_space4([300.0], cr.scalebroad, stride=4)
    assert np.all(est % 4 == 0)
    ratio = est.sum() / full.sum()
    assert 0.7 < ratio < 1.3


def test_force_constant_files_give_identical_rates(lib, tmp_path):
    """synthetic Phi3/Phi4 -> FORCE_CONSTANTS_3RD/4TH -> read back -> fp_init: three- and four-phonon rates equal to
    those of the in-memory force constants bit for bit."""
    cr = synth.diamond_si((3, 3, 2))
    w, e, v = oracle_modes(cr)
    p4, p3 = str(tmp_path / "FORCE_CONSTANTS_4TH"), str(tmp_path / "FORCE_CONSTANTS_3RD")
    lib.write_fc4(p4, cr.lattice, cr.fc4_idx, cr.fc4_val)
    lib.write_fc3(p3, cr.lattice, cr.fc3_idx, cr.fc3_val)
    fromfile = cr.with_grid(cr.grid)
    fromfile.fc4_idx, fromfile.fc4_val = lib.read_fc4(p4, cr.lattice)
    fromfile.fc3_idx, fromfile.fc3_val = lib.read_fc3(p3, cr.lattice)
    out = []
    for c in (cr, fromfile):
        with lib.Context.from_crystal(c) as ctx:
            ctx.set_modes(w, e, v)
            r4, st = ctx.rates4([300.0, 700.0], cr.scalebroad)
            r3, _ = ctx.rates3([300.0, 700.0], cr.scalebroad)
            out.append((r4, r3, st["accepted"]))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2] and out[0][0].max() > 0


def test_command_line_tasks(lib, tmp_path, capsys):
    from paper_2104_04895_gb300.__main__ import main
    fc = str(tmp_path / "FORCE_CONSTANTS_4TH")
    assert main(["onlyharmonic", "--workload", "1", "--temps", "300", "600", "--out", str(tmp_path / "ph"),
                 "--write-fc4", fc]) == 0
    ph = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert main(["rta", "--workload", "1", "--fc4", fc, "--out", str(tmp_path / "rta")]) == 0
    rta = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    cr = synth.workload(1)
    for name in ("BTE.omega", "BTE.Numprocess_4ph", "BTE.P4", "T300K/BTE.WP4", "T600K/BTE.WP4"):
        assert os.path.exists(tmp_path / "ph" / name)
    w, n = bte.read_mode_file(str(tmp_path / "ph" / "BTE.Numprocess_4ph"))
    assert w.shape == (cr.nq, cr.nb) and n.sum() == ph["processes"] > 0
    _, tot = bte.read_mode_file(str(tmp_path / "rta" / "T300K" / "BTE.w_4ph"))
    _, nor = bte.read_mode_file(str(tmp_path / "rta" / "T300K" / "BTE.w_4ph_normal"))
    _, umk = bte.read_mode_file(str(tmp_path / "rta" / "T300K" / "BTE.w_4ph_Umklapp"))
    np.testing.assert_allclose(nor + umk, tot, rtol=1e-12, atol=0.0)
    with lib.Context.from_crystal(cr) as ctx:
        ctx.modes(copy=False)
        direct, _ = ctx.rates4([300.0], cr.scalebroad)
    assert np.array_equal(tot, direct[0])
    assert rta["accepted"][1] > 0
