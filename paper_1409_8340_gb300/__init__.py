"""GB300-native implicit TDGL solver (arXiv:1409.8340).

Submodules: `solver` (Params, Solver, pattern), `presets` (named workloads),
`inputs` (seeded synthetic inputs), `build` (compiles libtdgl_gb300.so).
Nothing is loaded at import time; the CUDA library is loaded on first use and
its absence raises.
"""
