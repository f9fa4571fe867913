// Explicit instantiation of the 2D FFT passes for one group of line lengths.
#include "fft2d.cuh"
#include "internal.h"

#define EXT_INST(N) template struct FftOps<N>;
EXT_FFT_SIZES_E(EXT_INST)
