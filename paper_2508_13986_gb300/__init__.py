"""GB300-native GBEES: sparse-grid propagation of a probability density
(arXiv 2508.13986) in hand-written sm_103a CUDA behind a C ABI.

Submodules: `gbees` (the binding of include/gbees.h: one grid, or many in
one launch), `workloads` (seeded synthetic inputs), `build` (compiles the CUDA
library in-tree), `serving` (a continuous-batching request loop), `autotune`
(launch shapes chosen by measurement), `convergence` (E(t) and Bhattacharyya
coefficient studies in the CFL number and the cell width).
"""
