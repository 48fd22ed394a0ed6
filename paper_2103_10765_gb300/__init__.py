"""GB300 (sm_103a) implementation of the G-BM3D denoising hot path
(Sanders & Larkin, arXiv 2103.10765): block matching, stage-1 global 3-D
wavelet hard thresholding, stage-2 empirical Wiener filtering and weighted
aggregation, all as hand-written CUDA behind the C ABI of include/gbm3d.h.

Submodules: `gbm3d` is the Python binding (torch tensors in and out),
`synth` makes the seeded synthetic test images, `build` compiles the library.
"""
