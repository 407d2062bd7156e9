"""GB300-native four-phonon scattering rates (arXiv 2104.04895 hot path).

`binding` is the ctypes binding of the C-ABI library built from `csrc/` by `build`;
`synth` builds the seeded synthetic crystals used by the tests and the benchmark.
"""
__all__ = ["binding", "build", "synth"]
