"""Command-line runs of the library, after the paper's two tasks (Sec. 2.1, Appendix A):

  python -m paper_2104_04895_gb300 onlyharmonic --workload 2 --out run/     # phase space: Numprocess, P4, WP4
  python -m paper_2104_04895_gb300 rta --workload 2 --out run/              # RTA rates, normal and Umklapp parts
  python -m paper_2104_04895_gb300 rta --workload 5 --out run/ --checkpoint ck/ --slices 16 --no-nu-split
                                                                            # resumable: rerun after a stop

The crystal is one of the seeded synthetic workloads (paper_2104_04895_gb300.synth); --fc4 FILE replaces its
fourth-order force constants by those of a FORCE_CONSTANTS_4TH file (--fc3 likewise for the third order), and
--write-fc4 / --write-fc3 FILE write the crystal's force constants in that layout.  Everything runs on the GPU
through the C-ABI; the output files are described in paper_2104_04895_gb300.bte.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import binding, bte, resume, synth


def parse(argv):
    p = argparse.ArgumentParser(prog="python -m paper_2104_04895_gb300")
    p.add_argument("task", choices=["onlyharmonic", "rta"])
    p.add_argument("--workload", type=int, default=1, help="synthetic crystal 1-5")
    p.add_argument("--grid", type=int, nargs=3, default=None)
    p.add_argument("--temps", type=float, nargs="+", default=None)
    p.add_argument("--scalebroad", type=float, default=None)
    p.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    p.add_argument("--fc4", default=None, help="read the fourth-order force constants from this file")
    p.add_argument("--fc3", default=None, help="read the third-order force constants from this file")
    p.add_argument("--write-fc4", default=None, help="write the crystal's fourth-order force constants here")
    p.add_argument("--write-fc3", default=None, help="write the crystal's third-order force constants here")
    p.add_argument("--no-nu-split", action="store_true", help="rta: skip the normal/Umklapp parts")
    p.add_argument("--checkpoint", default=None,
                   help="rta: run the rates in slices of whole pairs {q, -q} with one checkpoint file per finished "
                        "slice in this directory; a rerun loads the finished slices (paper_2104_04895_gb300.resume)")
    p.add_argument("--slices", type=int, default=8, help="rta with --checkpoint: number of slices")
    p.add_argument("--device", type=int, default=0)
    p.add_argument("--out", required=True)
    return p.parse_args(argv)


def main(argv=None) -> int:
    a = parse(sys.argv[1:] if argv is None else argv)
    cr = synth.workload(a.workload)
    if a.grid:
        cr = cr.with_grid(a.grid)
    if a.temps:
        cr = cr.with_grid(cr.grid, temps=a.temps)
    if a.scalebroad is not None:
        cr.scalebroad = float(a.scalebroad)
    if a.fc4:
        cr.fc4_idx, cr.fc4_val = binding.read_fc4(a.fc4, cr.lattice)
    if a.fc3:
        cr.fc3_idx, cr.fc3_val = binding.read_fc3(a.fc3, cr.lattice)
    if a.write_fc4:
        binding.write_fc4(a.write_fc4, cr.lattice, cr.fc4_idx, cr.fc4_val)
    if a.write_fc3 and cr.fc3_idx is not None:
        binding.write_fc3(a.write_fc3, cr.lattice, cr.fc3_idx, cr.fc3_val)
    prec = binding.FP_PREC_FP64 if a.precision == "fp64" else binding.FP_PREC_MIXED
    temps = list(cr.temps)
    t0 = time.perf_counter()
    with binding.Context.from_crystal(cr, device=a.device) as ctx:
        w, _, _ = ctx.modes()
        if a.task == "onlyharmonic":
            npr, p4, wp4 = ctx.phase_space4(temps, cr.scalebroad, stride=1, precision=prec)
            paths = bte.write_phase_space(a.out, w, temps, npr, p4, wp4)
            summary = {"processes": float(np.sum(npr))}
        else:
            if a.checkpoint:
                rates, st = resume.rates4_resumable(ctx, temps, cr.scalebroad, a.checkpoint, a.slices,
                                                    precision=prec)
            else:
                rates, st = ctx.rates4(temps, cr.scalebroad, precision=prec)
            normal = umklapp = None
            if not a.no_nu_split:
                nu, _ = ctx.rates4_nu(temps, cr.scalebroad, precision=prec)
                normal, umklapp = nu[:, 0], nu[:, 1]
            paths = bte.write_rates(a.out, w, temps, rates, normal, umklapp)
            summary = {"accepted": st["accepted"], "candidates": st["candidates"]}
    summary.update({"task": a.task, "workload": cr.name, "grid": list(cr.grid), "temps": temps,
                    "seconds": time.perf_counter() - t0, "files": paths})
    print(json.dumps(summary))
    return 0


if __name__ == "__main__":
    sys.exit(main())
