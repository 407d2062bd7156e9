"""Oracle for the four-phonon scattering-rate path: TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg
may import this package.  It shares no code with the CUDA path (no kernels,
headers, helpers, tables or constants); both sides only read the seeded inputs
of `paper_2104_04895_gb300.synth`.

* `fp_oracle.c`  plain FP64 C (OpenMP) rates and vertices (Eqs. tao0, 4phgamma, V4; Sec. 2.4)
* `modes.py`     harmonic frequencies, eigenvectors, velocities (numpy / LAPACK)
* `brute.py`     supercell brute-force vertex for tiny grids
* `mlp.py`       FP64 forward/backward of the surrogate network (for gradient checks)

Every function is pinned by the `-m "not gpu"` tests in `tests/test_oracle_*.py`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def build(force: bool = False) -> str:
    """Compile fp_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP, no FP contraction)."""
    out_dir = os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "liboracle.so")
    src = os.path.join(_HERE, "fp_oracle.c")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-fno-fast-math", "-D_GNU_SOURCE", "-o", tmp, src, "-lm"])
        os.replace(tmp, so)
    return so


def lib():
    """The oracle library.  FP_ORACLE_LIB, when set, names another build of fp_oracle.c to load instead (the
    mutation tests use it to check that the pins fail on a deliberately broken copy of the oracle)."""
    global _LIB
    if _LIB is None:
        L = ctypes.CDLL(os.environ.get("FP_ORACLE_LIB") or build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.oracle_rates4.restype = ctypes.c_int
        L.oracle_rates4.argtypes = [ip, dp, ctypes.c_int, dp, ctypes.c_int, ip, dp, dp, dp, dp,
                                    ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int, ctypes.c_int, ip, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, dp, dp]
        L.oracle_rates3.restype = ctypes.c_int
        L.oracle_rates3.argtypes = [ip, dp, ctypes.c_int, dp, ctypes.c_int, ip, dp, dp, dp, dp, ctypes.c_int, dp,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int, ip,
                                    ctypes.c_int, ctypes.c_int, dp, dp]
        L.oracle_v3.restype = ctypes.c_int
        L.oracle_v3.argtypes = [ip, dp, ctypes.c_int, dp, ctypes.c_int, ip, dp, dp, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, dp, ctypes.POINTER(ctypes.c_int)]
        L.oracle_umklapp.restype = ctypes.c_int
        L.oracle_umklapp.argtypes = [ip, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.oracle_v4.restype = ctypes.c_int
        L.oracle_v4.argtypes = [ip, dp, ctypes.c_int, dp, ctypes.c_int, ip, dp, dp, ctypes.c_int,
                                ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ip]
        L.oracle_phase3.restype = ctypes.c_int
        L.oracle_phase3.argtypes = [ip, dp, ctypes.c_int, dp, dp, ctypes.c_int, dp, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int, ip, dp, dp]
        L.oracle_bose.restype = ctypes.c_double
        L.oracle_bose.argtypes = [ctypes.c_double, ctypes.c_double]
        L.oracle_prefactor.restype = ctypes.c_double
        L.oracle_prefactor.argtypes = [ctypes.c_int]
        _LIB = L
    return _LIB


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def evec_to_array(ev):
    """complex (N, nb, nb) -> float (N, nb, nb, 2)"""
    return np.ascontiguousarray(np.stack([ev.real, ev.imag], axis=-1))


def rates4(cryst, omega, evec, vel, temps=None, scalebroad=None, window=2.0, sigma_min=1e-10, dq_mode=0,
           sel=None, unit_vertex=False, nthreads=0, processes=(0, 1, 2), nu=None):
    """Rates (nT, nsel) in ps^-1 and accepted counts (3,) for modes sel (default: all).

    unit_vertex: False/0 the rates; True/1 |V|^2 := 1 (weighted phase space WP4, sum without prefactor and 1/N^2);
    2 also Bose and frequency factors := 1 (phase space P4: sum of c_p delta_p).

    processes: the classes of Eq. 4phgamma summed, 0 ++ (recombination), 1 +- (redistribution), 2 --
    (splitting); the default sums all three (the full rate).  nu: None (all), "normal" or "umklapp" (Sec. 2.2,
    Q = 0 or not; the reading is in fp_oracle.c at orc_bz_shift)."""
    nu_select = {None: 0, "normal": 1, "umklapp": 2}[nu]
    temps = cryst.temps if temps is None else temps
    sb = cryst.scalebroad if scalebroad is None else scalebroad
    nb = cryst.nb
    N = cryst.nq
    if sel is None:
        sel = np.arange(N * nb)
    sel_a, sel_p = _i(np.asarray(sel))
    grid, grid_p = _i(np.asarray(cryst.grid))
    lat, lat_p = _d(cryst.lattice)
    m, m_p = _d(cryst.mass)
    qi, qi_p = _i(cryst.fc4_idx)
    qf, qf_p = _d(cryst.fc4_val)
    om, om_p = _d(omega)
    ev, ev_p = _d(evec_to_array(evec) if np.iscomplexobj(evec) else evec)
    ve, ve_p = _d(vel)
    T, T_p = _d(np.asarray(temps, float))
    out = np.zeros((len(temps), len(sel_a)))
    acc = np.zeros(3)
    _, out_p = _d(out)
    out_p = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    acc_p = acc.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    rc = lib().oracle_rates4(grid_p, lat_p, cryst.natoms, m_p, len(qi), qi_p, qf_p, om_p, ev_p, ve_p,
                             len(T), T_p, float(sb), float(window), float(sigma_min), int(dq_mode),
                             len(sel_a), sel_p, int(unit_vertex), sum(1 << int(p) for p in set(processes)),
                             nu_select, int(nthreads), out_p, acc_p)
    if rc != 0:
        raise ValueError("oracle_rates4 rejected its arguments")
    return out, acc


def v4(cryst, evec, q, q1, q2, process):
    """Branch tensor V[j, j1, j2, j3] (complex) of process 0:++, 1:+-, 2:-- and q'''."""
    nb = cryst.nb
    grid, grid_p = _i(np.asarray(cryst.grid))
    lat, lat_p = _d(cryst.lattice)
    m, m_p = _d(cryst.mass)
    qi, qi_p = _i(cryst.fc4_idx)
    qf, qf_p = _d(cryst.fc4_val)
    ev, ev_p = _d(evec_to_array(evec) if np.iscomplexobj(evec) else evec)
    out = np.zeros((nb, nb, nb, nb, 2))
    q3 = ctypes.c_int(0)
    rc = lib().oracle_v4(grid_p, lat_p, cryst.natoms, m_p, len(qi), qi_p, qf_p, ev_p, int(q), int(q1), int(q2),
                         int(process), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(q3))
    if rc != 0:
        raise ValueError("oracle_v4 rejected its arguments")
    return out[..., 0] + 1j * out[..., 1], q3.value


def phase3(cryst, omega, vel, temps=None, scalebroad=None, window=2.0, sigma_min=1e-10, dq_mode=0, sel=None):
    """Three-phonon-like phase space P3 (nsel,) and weighted WP3 (nT, nsel) of modes sel (default all)."""
    temps = cryst.temps if temps is None else temps
    sb = cryst.scalebroad if scalebroad is None else scalebroad
    if sel is None:
        sel = np.arange(cryst.nq * cryst.nb)
    sel_a, sel_p = _i(np.asarray(sel))
    grid, grid_p = _i(np.asarray(cryst.grid))
    lat, lat_p = _d(cryst.lattice)
    om, om_p = _d(omega)
    ve, ve_p = _d(vel)
    T, T_p = _d(np.asarray(temps, float))
    p3 = np.zeros(len(sel_a))
    wp3 = np.zeros((len(T), len(sel_a)))
    rc = lib().oracle_phase3(grid_p, lat_p, cryst.natoms, om_p, ve_p, len(T), T_p, float(sb), float(window),
                             float(sigma_min), int(dq_mode), len(sel_a), sel_p,
                             p3.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             wp3.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise ValueError("oracle_phase3 rejected its arguments")
    return p3, wp3


def bose(w, T):
    return lib().oracle_bose(float(w), float(T))


def prefactor(nq):
    return lib().oracle_prefactor(int(nq))


def umklapp(cryst, q, q1, q2, process):
    """1 if process (0 ++, 1 +-, 2 --) with partners q1, q2 of mode wavevector q is Umklapp, 0 if normal."""
    grid, grid_p = _i(np.asarray(cryst.grid))
    lat, lat_p = _d(cryst.lattice)
    r = lib().oracle_umklapp(grid_p, lat_p, int(q), int(q1), int(q2), int(process))
    if r < 0:
        raise ValueError("oracle_umklapp rejected its arguments")
    return r


def rates3(cryst, omega, evec, vel, temps=None, scalebroad=None, window=2.0, sigma_min=1e-10, dq_mode=0, sel=None,
           unit_vertex=False, nthreads=0):
    """Three-phonon RTA rates (nT, nsel) in ps^-1 (Eqs. tao0, 3phgamma, V3) and accepted counts (+, -)."""
    temps = cryst.temps if temps is None else temps
    sb = cryst.scalebroad if scalebroad is None else scalebroad
    nb, N = cryst.nb, cryst.nq
    if sel is None:
        sel = np.arange(N * nb)
    sel_a, sel_p = _i(np.asarray(sel))
    grid, grid_p = _i(np.asarray(cryst.grid))
    lat, lat_p = _d(cryst.lattice)
    m, m_p = _d(cryst.mass)
    qi, qi_p = _i(cryst.fc3_idx)
    qf, qf_p = _d(cryst.fc3_val)
    om_, om_p = _d(omega)
    ev, ev_p = _d(evec_to_array(evec) if np.iscomplexobj(evec) else evec)
    ve, ve_p = _d(vel)
    T, T_p = _d(np.asarray(temps, float))
    out = np.zeros((len(temps), len(sel_a)))
    acc = np.zeros(2)
    rc = lib().oracle_rates3(grid_p, lat_p, cryst.natoms, m_p, len(qi), qi_p, qf_p, om_p, ev_p, ve_p, len(T), T_p,
                             float(sb), float(window), float(sigma_min), int(dq_mode), len(sel_a), sel_p,
                             int(bool(unit_vertex)), int(nthreads), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             acc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise ValueError("oracle_rates3 rejected its arguments")
    return out, acc


def v3(cryst, evec, q, q1, process):
    """Branch tensor V[j, j1, j2] (complex) of process 0 (+) or 1 (-) with partner q1, and q''."""
    nb = cryst.nb
    grid, grid_p = _i(np.asarray(cryst.grid))
    lat, lat_p = _d(cryst.lattice)
    m, m_p = _d(cryst.mass)
    qi, qi_p = _i(cryst.fc3_idx)
    qf, qf_p = _d(cryst.fc3_val)
    ev, ev_p = _d(evec_to_array(evec) if np.iscomplexobj(evec) else evec)
    out = np.zeros((nb, nb, nb, 2))
    q2 = ctypes.c_int(0)
    rc = lib().oracle_v3(grid_p, lat_p, cryst.natoms, m_p, len(qi), qi_p, qf_p, ev_p, int(q), int(q1), int(process),
                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(q2))
    if rc != 0:
        raise ValueError("oracle_v3 rejected its arguments")
    return out[..., 0] + 1j * out[..., 1], q2.value


# CODATA 2018 constants in the units of the rates (the same data as fp_oracle.c's ORC_HBAR / ORC_KB)
_HBAR_EV_PS = 6.582119569e-4
_KB_EV_K = 8.617333262e-5
_KB_J_K = 1.380649e-23


def kappa_rta(lattice, omega, vel, temps, rates):
    """RTA lattice thermal conductivity (nT, 3, 3) in W/(m K), the kinetic form that the rates feed:
    kappa_ab = k_B / (N V) sum_modes c(x) v_a v_b / rate, c(x) = x^2 e^x / (e^x - 1)^2, x = hbar w / (k_B T).
    omega (N, nb) rad/ps, vel (N, nb, 3) A/ps, rates (nT, N, nb) ps^-1; modes with w = 0 or rate <= 0 are left out.
    Units: k_B [J/K] (A/ps)^2 ps / A^3 = k_B * 1e4 * 1e-12 / 1e-30 W/(m K)."""
    w = np.asarray(omega, float).reshape(-1)
    v = np.asarray(vel, float).reshape(-1, 3)
    r = np.asarray(rates, float).reshape(len(temps), -1)
    N = np.asarray(omega).shape[0]
    V = abs(np.linalg.det(np.asarray(lattice, float)))
    out = np.zeros((len(temps), 3, 3))
    for t, T in enumerate(temps):
        for m in range(len(w)):
            if not (w[m] > 0.0 and r[t, m] > 0.0):
                continue
            x = _HBAR_EV_PS * w[m] / (_KB_EV_K * T)
            c = x * x * np.exp(x) / np.expm1(x) ** 2
            out[t] += c / r[t, m] * np.outer(v[m], v[m])
    return out * _KB_J_K * 1e4 * 1e-12 / 1e-30 / (N * V)
