"""GB300-native brushed multivariate volume rendering (arXiv 2207.12011).

`paper_2207_12011_gb300.raypc` is the Python binding of the C-ABI library
`libraypc.so` (CUDA kernels for sm_103a); `paper_2207_12011_gb300.synth`
generates seeded synthetic workloads. The binding loads the library on first
use and raises if it is missing: there is no CPU fallback.
"""
