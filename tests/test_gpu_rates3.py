"""GPU three-phonon rates (fp_set_fc3 / fp_rates3) against the FP64 oracle, through the C-ABI.

Modes are injected from the oracle, so window decisions must agree exactly (accepted counts compared as
integers) and the rates to 1e-10 relative."""
import numpy as np
import pytest

import oracle
from paper_2104_04895_gb300 import synth

from conftest import oracle_modes

pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module")
def lib():
    from paper_2104_04895_gb300 import binding
    binding.load()
    return binding


def compare(gpu, ref):
    gpu, ref = np.asarray(gpu), np.asarray(ref)
    zero = ref == 0.0
    assert np.all(gpu[zero] == 0.0)
    rel = np.abs(gpu[~zero] - ref[~zero]) / np.abs(ref[~zero])
    assert rel.max(initial=0.0) <= RTOL, f"max rel err {rel.max():.3e}"


CASES = [("sc-4x4x4", lambda: synth.simple_cubic((4, 4, 4))), ("diamond-3x3x2", lambda: synth.diamond_si((3, 3, 2))),
         ("bas-3x3x3", lambda: synth.zincblende_bas((3, 3, 3))), ("licoo2-3x3x2", lambda: synth.licoo2((3, 3, 2)))]


@pytest.mark.parametrize("name,maker", CASES, ids=[c[0] for c in CASES])
def test_rates3_parity(lib, name, maker):
    cr = maker()
    w, e, v = oracle_modes(cr)
    temps = [300.0, 700.0]
    ref, acc = oracle.rates3(cr, w, e, v, temps=temps)
    with lib.Context.from_crystal(cr) as ctx:
        ctx.set_modes(w, e, v)
        out, st = ctx.rates3(temps, cr.scalebroad)
    compare(out.reshape(len(temps), -1), ref)
    assert st["accepted"][:2] == list(acc) and st["accepted"][2] == 0
    assert st["candidates"] == 2.0 * cr.nq * cr.nb * cr.nq * cr.nb ** 2


def test_rates3_options(lib):
    cr = synth.diamond_si((3, 3, 2))
    w, e, v = oracle_modes(cr)
    nb = cr.nb
    rng = np.random.Generator(np.random.PCG64(33))
    mask = (rng.random(cr.nq * nb) < 0.4).astype(np.uint8)
    sel = np.nonzero(mask)[0]
    with lib.Context.from_crystal(cr) as ctx:
        ctx.set_modes(w, e, v)
        out, _ = ctx.rates3(cr.temps, cr.scalebroad, mode_mask=mask, dq_mode=1, window=3.0)
        rq, _ = ctx.rates3(cr.temps, cr.scalebroad, q_begin=4, q_end=9)
    ref, _ = oracle.rates3(cr, w, e, v, sel=sel, dq_mode=1, window=3.0)
    flat = out.reshape(-1)
    compare(flat[sel][None, :], ref)
    assert np.all(flat[mask == 0] == 0.0)
    sel = np.arange(4 * nb, 9 * nb)
    ref, _ = oracle.rates3(cr, w, e, v, sel=sel)
    flat = rq.reshape(-1)
    compare(flat[sel][None, :], ref)
    assert np.all(flat[:4 * nb] == 0.0) and np.all(flat[9 * nb:] == 0.0)


def test_rates3_full_size_sampled(lib):
    """Diamond 8x8x8: the full grid on the GPU, three sampled modes against the oracle."""
    cr = synth.workload(2)
    w, e, v = oracle_modes(cr)
    with lib.Context.from_crystal(cr) as ctx:
        ctx.set_modes(w, e, v)
        out, st = ctx.rates3(cr.temps, cr.scalebroad)
    rng = np.random.Generator(np.random.PCG64(2104))
    sel = np.sort(rng.choice(np.arange(cr.nb, cr.nq * cr.nb), size=3, replace=False))
    ref, _ = oracle.rates3(cr, w, e, v, sel=sel)
    compare(out.reshape(1, -1)[:, sel], ref)
    print(f"diamond 8^3 three-phonon rates: {st['ms']:.1f} ms, {st['candidates'] / st['ms'] * 1e3:.3e} terms/s")


def test_rates3_needs_fc3(lib):
    cr = synth.simple_cubic((2, 2, 2))
    w, e, v = oracle_modes(cr)
    with lib.Context(cr.lattice, cr.frac, cr.mass, cr.fc2_idx, cr.fc2_val, cr.fc4_idx, cr.fc4_val, cr.grid) as ctx:
        ctx.set_modes(w, e, v)
        with pytest.raises(lib.FourPhononError) as ei:
            ctx.rates3(cr.temps, cr.scalebroad)
        assert ei.value.code == lib.FP_ESTATE


def test_kappa_rta_matches_the_oracle(lib):
    """fp_kappa_rta on the GPU rates (three- plus four-phonon) equals the oracle's kinetic form on the same
    rates and modes."""
    cr = synth.diamond_si((3, 3, 2))
    w, e, v = oracle_modes(cr)
    temps = [300.0, 600.0]
    with lib.Context.from_crystal(cr) as ctx:
        ctx.set_modes(w, e, v)
        r3, _ = ctx.rates3(temps, cr.scalebroad)
        r4, _ = ctx.rates4(temps, cr.scalebroad)
        k = ctx.kappa_rta(temps, r3 + r4)
        with pytest.raises(lib.FourPhononError):
            ctx.kappa_rta([0.0], r3[:1])
    ref = oracle.kappa_rta(cr.lattice, w, v, temps, r3 + r4)
    np.testing.assert_allclose(k, ref, rtol=1e-11, atol=1e-14 * np.abs(ref).max())
    assert np.all(np.diagonal(k, axis1=1, axis2=2) > 0.0)
    print(f"diamond 3x3x2 kappa_xx: {k[0, 0, 0]:.4g} W/mK (300 K), {k[1, 0, 0]:.4g} W/mK (600 K)")
