"""GB300-native (sm_103a) half-space Spectral Ewald summation for Stokes flow.

Implements the fast Ewald method of Srinivasan & Tornberg (arXiv 1802.07844)
for stokeslet, stresslet and rotlet sums above a no-slip wall: a real-space
erfc-screened neighbour sum over sources and wall images, and a Fourier-space
part (Gaussian spreading, zero-padded 3-D FFT, scaling by truncated kernels,
inverse FFT, Gaussian quadrature), all in hand-written CUDA kernels behind the
C ABI of ``include/hse.h``.  FP64 plans run the real-space pairs within rc64 in
FP64 (an outer shell in FP32) and the Fourier part in double-float arithmetic
with the library's own zero-padded transforms (cuFFT double on request or
below tol 1e-12); mixed-precision plans run FP32 arithmetic with cuFFT single.

``hse`` is the ctypes binding; ``build`` compiles the library in-tree.
"""
from .hse import (HSE_FFT_AUTO, HSE_FFT_CUFFT, HSE_FFT_DF64, HSE_FP64, HSE_FREE_SPACE, HSE_MIXED, HSE_ROTLET, HSE_STOKESLET, HSE_STRESSLET, Batch, HseError, Plan,  # noqa: F401
                  hse_cell_list, hse_eval, hse_eval_parts, hse_get_eval_stats, hse_plan_set_timing, hse_neighbor_counts, hse_plan_create,
                  hse_plan_destroy, hse_plan_get_params, hse_plan_set_fft, hse_plan_set_grid, hse_spread_grids, load)
