// pol2.cu - total power of two recorded polarisations (Section 2: the FAST
// data record two; Eq. 1's B is the total power).
//
// With x_a = p0_a + p1_a, sum_t x_a x_b is the sum of the four
// polarisation products sum p0_a p0_b + p0_a p1_b + p1_a p0_b + p1_a p1_b,
// and sum_t x_a = sum p0_a + sum p1_a. So the exact Gram of the total power
// is a fold of the exact Gram of the 2N stacked polarisation blocks (block
// p*N + a = polarisation p of beam a), which the 8-bit Gram kernels form
// as they stand; int64 addition keeps it exact. (Where the tensor-core Gram
// takes the shape it adds the polarisations itself and needs none of this.)
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace mraid {
namespace {

// out [cell][P], P = (N+1)(N+2)/2, from in [cell][P2], P2 = (2N+1)(2N+2)/2;
// both packed upper triangles, row-major.
__global__ void pol2_fold_kernel(const int64_t* __restrict__ in, int64_t* __restrict__ out,
                                 int64_t n_cells, int N, int P, int P2) {
  const int M2 = 2 * N + 1;
  const int64_t total = n_cells * P;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = idx / P;
    int e = (int)(idx - cell * P);
    int a = 0;
    while (e >= N + 1 - a) {  // row a of the (N+1)-triangle holds N + 1 - a entries
      e -= N + 1 - a;
      ++a;
    }
    const int b = a + e;
    const int64_t* S = in + cell * P2;
    auto at = [&](int i, int j) {  // entry (i, j) of the stacked Gram, any order
      if (i > j) {
        const int t = i;
        i = j;
        j = t;
      }
      return S[i * M2 - i * (i - 1) / 2 + (j - i)];
    };
    int64_t v;
    if (a == N) v = at(2 * N, 2 * N);                          // n
    else if (b == N) v = at(a, 2 * N) + at(a + N, 2 * N);      // sum x_a
    else v = at(a, b) + at(a, b + N) + at(a + N, b) + at(a + N, b + N);
    out[idx] = v;
  }
}

}  // namespace

cudaError_t launch_pol2_fold(const mraid_plan_s* pl, const int64_t* d_stacked, int64_t n_cells,
                             int64_t* d_sums) {
  const int N = pl->p.n_beam;
  const int P = pl->psum, P2 = (2 * N + 1) * (2 * N + 2) / 2;
  const int64_t total = n_cells * P;
  int64_t blocks = (total + 255) / 256;
  if (blocks > (int64_t)pl->sm_count * 16) blocks = (int64_t)pl->sm_count * 16;
  if (blocks < 1) return cudaSuccess;
  pol2_fold_kernel<<<(unsigned)blocks, 256, 0, pl->stream>>>(d_stacked, d_sums, n_cells, N, P, P2);
  return cudaGetLastError();
}

}  // namespace mraid
