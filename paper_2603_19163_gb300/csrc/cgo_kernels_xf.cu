// The single-solve kernels with island migration and crossover compiled in
// (evolve_kernel<..., XF = true>).  They are the same templates as in
// cgo_kernels.cu, instantiated in a translation unit of their own so that
// the two kernel sets compile in parallel.
#define CGO_XF_UNIT 1
#include "cgo_kernels.cu"
