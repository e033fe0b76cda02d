// Column-block copies of the prognostic state for the x-y pencil decomposition: the halo strips
// one rank sends to its neighbours once per RK3 step.  A block is the columns [i0, i0+ni) x
// [j0, j0+nj) at every level of one field, packed [k][jj][ii] (ii fastest), so a warp reads and
// writes consecutive x positions of one row.  The state keeps its storage type (FP64, or the FP32
// perturbations of the mixed path): a copied block is bit-identical to its source.
#include <cuda_runtime.h>

#include "erf_launch.h"

namespace erfk {

template <typename T>
__global__ void k_column_block(T *field, T *buf, int nx, int ny, int levels, int i0, int ni, int j0, int nj,
                               int unpack) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long per_level = (long long)ni * nj;
    if (t >= per_level * levels) return;
    const int ii = (int)(t % ni);
    const long long r = t / ni;
    const int jj = (int)(r % nj), k = (int)(r / nj);
    const long long f = ((long long)k * ny + (j0 + jj)) * nx + (i0 + ii);
    if (unpack) field[f] = buf[t];
    else buf[t] = field[f];
}

void launch_column_block(void *field, void *buf, int elem_bytes, int nx, int ny, int levels, int i0, int ni,
                         int j0, int nj, int unpack, cudaStream_t s) {
    const long long n = (long long)ni * nj * levels;
    if (n <= 0) return;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (elem_bytes == 8)
        k_column_block<double><<<blocks, 256, 0, s>>>((double *)field, (double *)buf, nx, ny, levels, i0, ni, j0,
                                                      nj, unpack);
    else
        k_column_block<float><<<blocks, 256, 0, s>>>((float *)field, (float *)buf, nx, ny, levels, i0, ni, j0,
                                                     nj, unpack);
}

}  // namespace erfk
