"""GPU harmonic modes (fp_modes) vs the oracle, and the C-ABI's error behaviour."""
import numpy as np
import pytest

import oracle
import oracle.modes as om
from paper_2104_04895_gb300 import synth
from paper_2104_04895_gb300.binding import FP_EINVAL, FP_ESTATE, FourPhononError

from conftest import oracle_modes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2104_04895_gb300 import binding
    binding.load()
    return binding


@pytest.mark.parametrize("maker", [lambda: synth.workload(1), lambda: synth.diamond_si((4, 4, 4)),
                                   lambda: synth.licoo2((3, 3, 2)), lambda: synth.zincblende_bas((3, 3, 3))])
def test_modes_match_oracle(lib, maker):
    cr = maker()
    w0, e0, v0 = oracle_modes(cr)
    with lib.Context.from_crystal(cr) as ctx:
        w, e, v = ctx.modes()
    np.testing.assert_allclose(w, w0, rtol=1e-10, atol=1e-9)
    G = om.grid_points(cr.grid)
    ng = np.array(cr.grid)
    for q in range(cr.nq):
        p = int(np.ravel_multi_index(tuple((-G[q]) % ng), cr.grid))
        assert np.array_equal(w[p], w[q]) and np.array_equal(e[p], e[q].conj()) and np.array_equal(v[p], -v[q])
        # gauge-invariant comparison: projector on each degenerate set, and set-averaged velocities
        for (b, en) in om.degenerate_sets(w0[q]):
            P = e[q, b:en].T @ e[q, b:en].conj()
            P0 = e0[q, b:en].T @ e0[q, b:en].conj()
            assert np.abs(P - P0).max() < 1e-8
            np.testing.assert_allclose(v[q, b:en], v0[q, b:en], rtol=1e-8, atol=1e-8 * max(1.0, np.abs(v0).max()))


def test_whole_path_with_gpu_modes(lib):
    """fp_modes + fp_rates4 against oracle modes + oracle rates, degenerate-set averaged."""
    cr = synth.workload(1)
    w0, e0, v0 = oracle_modes(cr)
    ref, _ = oracle.rates4(cr, w0, e0, v0)
    with lib.Context.from_crystal(cr) as ctx:
        w, e, v = ctx.modes()
        out, _ = ctx.rates4(cr.temps, cr.scalebroad)
    ref = ref.reshape(cr.nq, cr.nb)
    out = out.reshape(cr.nq, cr.nb)
    for q in range(cr.nq):
        for (b, en) in om.degenerate_sets(w0[q]):
            a, r = out[q, b:en].mean(), ref[q, b:en].mean()
            assert a == pytest.approx(r, rel=1e-6, abs=1e-14)


def test_errors(lib):
    cr = synth.simple_cubic((2, 2, 2))
    with pytest.raises(FourPhononError) as ei:
        lib.Context(cr.lattice, cr.frac, -cr.mass, cr.fc2_idx, cr.fc2_val, cr.fc4_idx, cr.fc4_val, cr.grid)
    assert ei.value.code == FP_EINVAL
    bad = cr.fc4_idx.copy()
    bad[0, 2] = 5
    with pytest.raises(FourPhononError) as ei:
        lib.Context(cr.lattice, cr.frac, cr.mass, cr.fc2_idx, cr.fc2_val, bad, cr.fc4_val, cr.grid)
    assert ei.value.code == FP_EINVAL
    with lib.Context.from_crystal(cr) as ctx:
        with pytest.raises(FourPhononError) as ei:
            ctx.rates4([300.0])
        assert ei.value.code == FP_ESTATE
        w, e, v = oracle_modes(cr)
        e2 = e.copy()
        e2[1] = e2[1] * 1j  # breaks e(-q) = conj e(q)
        with pytest.raises(FourPhononError) as ei:
            ctx.set_modes(w, e2, v)
        assert ei.value.code == FP_EINVAL
        ctx.set_modes(w, e, v)
        for kw in (dict(temps=[-1.0]), dict(temps=[300.0], scalebroad=0.0)):
            with pytest.raises(FourPhononError) as ei:
                ctx.rates4(**kw)
            assert ei.value.code == FP_EINVAL
        with pytest.raises(FourPhononError) as ei:
            ctx.rates4([300.0], block_j0=2)  # does not divide nb = 3
        assert ei.value.code == FP_EINVAL
        out, _ = ctx.rates4([300.0])   # the context is still usable after rejected calls
        assert np.all(np.isfinite(out))


def test_injected_allocation_failure_is_reported_and_recoverable(lib, monkeypatch):
    """FP_FAULT_ALLOC=k makes the k-th device allocation report out-of-memory (host-side injection)."""
    from paper_2104_04895_gb300.binding import FP_ENOMEM
    cr = synth.simple_cubic((2, 2, 2))
    for k in (1, 3, 7):
        monkeypatch.setenv("FP_FAULT_ALLOC", str(k))
        with pytest.raises(FourPhononError) as ei:
            lib.Context.from_crystal(cr)
        assert ei.value.code == FP_ENOMEM
        monkeypatch.delenv("FP_FAULT_ALLOC")
    with lib.Context.from_crystal(cr) as ctx:   # nothing leaked or left broken
        w, e, v = oracle_modes(cr)
        ctx.set_modes(w, e, v)
        out, _ = ctx.rates4([300.0])
        assert np.all(np.isfinite(out))
