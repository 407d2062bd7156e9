"""Force-constant files (FORCE_CONSTANTS_3RD / 4TH layout, Appendix A) and the BTE.* output files, on the CPU:
the library's reader returns exactly what its writer wrote, and malformed files are rejected with a message."""
import os

import numpy as np
import pytest

from paper_2104_04895_gb300 import binding, bte, synth


@pytest.mark.parametrize("wl", [1, 2, 3, 4])
def test_round_trip_is_bit_exact(tmp_path, wl):
    cr = synth.workload(wl)
    p4 = str(tmp_path / "FORCE_CONSTANTS_4TH")
    p3 = str(tmp_path / "FORCE_CONSTANTS_3RD")
    binding.write_fc4(p4, cr.lattice, cr.fc4_idx, cr.fc4_val)
    binding.write_fc3(p3, cr.lattice, cr.fc3_idx, cr.fc3_val)
    i4, v4 = binding.read_fc4(p4, cr.lattice)
    i3, v3 = binding.read_fc3(p3, cr.lattice)
    assert np.array_equal(i4, cr.fc4_idx) and np.array_equal(v4, cr.fc4_val)
    assert np.array_equal(i3, cr.fc3_idx) and np.array_equal(v3, cr.fc3_val)
    lines = open(p4).read().split("\n")
    assert int(lines[0]) == len(cr.fc4_idx) and lines[1] == "" and lines[2] == "1"
    # block 1: three cell positions, four 1-based atom indices, then 81 value lines
    assert len(lines[6].split()) == 4 and all(len(x.split()) == 5 for x in lines[7:88])


def _write(path, text):
    with open(path, "w") as f:
        f.write(text)


def test_malformed_files_are_rejected(tmp_path):
    cr = synth.simple_cubic((1, 1, 1))
    good = str(tmp_path / "good")
    binding.write_fc4(good, cr.lattice, cr.fc4_idx[:1], cr.fc4_val[:1])
    text = open(good).read()
    lines = text.split("\n")
    off = lines[:]
    off[3] = "1.5 0 0"          # the first cell position, half a lattice vector away
    cases = {
        "not-a-lattice-vector": "\n".join(off),
        "repeated-index": text.replace("1 1 1 2 ", "1 1 1 1 ", 1),
        "truncated": "\n".join(text.split("\n")[:40]),
        "bad-count": "x\n" + text,
        "atom-0": text.replace("1 1 1 1\n", "0 1 1 1\n", 1),
    }
    for name, t in cases.items():
        p = str(tmp_path / name)
        _write(p, t)
        with pytest.raises(binding.FourPhononError):
            binding.read_fc4(p, cr.lattice)
        assert binding.load().fp_last_error(None)
    with pytest.raises(binding.FourPhononError):
        binding.read_fc4(str(tmp_path / "missing"), cr.lattice)


def test_count_query_and_short_buffer(tmp_path):
    import ctypes
    cr = synth.workload(2)
    p = str(tmp_path / "fc4")
    binding.write_fc4(p, cr.lattice, cr.fc4_idx, cr.fc4_val)
    L = binding.load()
    lat = np.ascontiguousarray(cr.lattice, np.float64).reshape(9)
    n = ctypes.c_int(0)
    assert L.fp_read_fc4(p.encode(), lat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None, 0,
                         ctypes.byref(n)) == binding.FP_OK
    assert n.value == len(cr.fc4_idx)
    arr = (binding.fp_fc4 * 3)()
    assert L.fp_read_fc4(p.encode(), lat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), arr, 3,
                         ctypes.byref(n)) == binding.FP_EINVAL


def test_bte_mode_files_round_trip(tmp_path):
    rng = np.random.Generator(np.random.PCG64(3))
    w = rng.uniform(0.0, 80.0, size=(7, 6))
    temps = [300.0, 650.0]
    npr = rng.integers(0, 10**9, size=42).astype(float)
    p4 = rng.random(42)
    wp4 = rng.random((2, 42))
    paths = bte.write_phase_space(str(tmp_path), w, temps, npr, p4, wp4)
    names = sorted(os.path.relpath(p, tmp_path) for p in paths)
    assert names == ["BTE.Numprocess_4ph", "BTE.P4", "BTE.omega", "T300K/BTE.WP4", "T650K/BTE.WP4"]
    w2, n2 = bte.read_mode_file(str(tmp_path / "BTE.Numprocess_4ph"))
    assert np.array_equal(w2, w) and np.array_equal(n2.reshape(-1), npr)
    _, x = bte.read_mode_file(str(tmp_path / "T650K" / "BTE.WP4"))
    assert np.array_equal(x.reshape(-1), wp4[1])
    r = rng.random((2, 7, 6))
    paths = bte.write_rates(str(tmp_path / "rta"), w, temps, r, 0.25 * r, 0.75 * r)
    assert len(paths) == 6
    _, u = bte.read_mode_file(str(tmp_path / "rta" / "T300K" / "BTE.w_4ph_Umklapp"))
    assert np.array_equal(u, 0.75 * r[0])
