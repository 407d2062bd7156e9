"""Output files of a four-phonon run, named as the paper's program names them (Appendix A).

Temperature-independent quantities go to the output directory, temperature-dependent ones to a subdirectory
``T<temperature>K`` per temperature.  Each file has one row per mode, q-major then branch (the library's mode
order): ``q j omega value`` with omega in rad/ps.

  BTE.omega            omega (rad/ps)
  BTE.Numprocess_4ph   number of allowed four-phonon processes of each mode
  BTE.P4               four-phonon phase space (ps)
  T*/BTE.WP4           weighted four-phonon phase space (ps^4)
  T*/BTE.w_4ph         four-phonon RTA scattering rate (1/ps)
  T*/BTE.w_4ph_normal  its normal-process part
  T*/BTE.w_4ph_Umklapp its Umklapp part

Formatting only; the numbers come from the library (fp_phase_space4, fp_rates4, fp_rates4_nu).
"""
from __future__ import annotations

import os

import numpy as np


def temperature_dir(outdir: str, T: float) -> str:
    d = os.path.join(outdir, f"T{T:g}K")
    os.makedirs(d, exist_ok=True)
    return d


def write_mode_file(path: str, omega, values) -> None:
    """Rows "q j omega value" for every mode; omega (N, nb), values (N*nb,) or (N, nb)."""
    w = np.asarray(omega, np.float64)
    N, nb = w.shape
    v = np.asarray(values, np.float64).reshape(N, nb)
    with open(path, "w") as f:
        for q in range(N):
            for j in range(nb):
                f.write(f"{q} {j} {w[q, j]:.17g} {v[q, j]:.17g}\n")


def read_mode_file(path: str):
    """(omega (N, nb), values (N, nb)) from a file of write_mode_file."""
    a = np.loadtxt(path, ndmin=2)
    N = int(a[:, 0].max()) + 1
    nb = int(a[:, 1].max()) + 1
    return a[:, 2].reshape(N, nb), a[:, 3].reshape(N, nb)


def write_phase_space(outdir: str, omega, temps, numprocess, p4, wp4) -> list[str]:
    """BTE.omega, BTE.Numprocess_4ph, BTE.P4 and T*/BTE.WP4; returns the paths written."""
    os.makedirs(outdir, exist_ok=True)
    paths = [os.path.join(outdir, "BTE.omega"), os.path.join(outdir, "BTE.Numprocess_4ph"),
             os.path.join(outdir, "BTE.P4")]
    w = np.asarray(omega)
    write_mode_file(paths[0], w, w)
    write_mode_file(paths[1], w, numprocess)
    write_mode_file(paths[2], w, p4)
    wp4 = np.asarray(wp4).reshape(len(temps), -1)
    for t, T in enumerate(temps):
        p = os.path.join(temperature_dir(outdir, T), "BTE.WP4")
        write_mode_file(p, w, wp4[t])
        paths.append(p)
    return paths


def write_rates(outdir: str, omega, temps, rates, normal=None, umklapp=None) -> list[str]:
    """T*/BTE.w_4ph and, when given, T*/BTE.w_4ph_normal and T*/BTE.w_4ph_Umklapp; returns the paths written."""
    os.makedirs(outdir, exist_ok=True)
    w = np.asarray(omega)
    paths = []
    parts = [("BTE.w_4ph", rates), ("BTE.w_4ph_normal", normal), ("BTE.w_4ph_Umklapp", umklapp)]
    for t, T in enumerate(temps):
        d = temperature_dir(outdir, T)
        for name, arr in parts:
            if arr is None:
                continue
            p = os.path.join(d, name)
            write_mode_file(p, w, np.asarray(arr).reshape(len(temps), -1)[t])
            paths.append(p)
    return paths
