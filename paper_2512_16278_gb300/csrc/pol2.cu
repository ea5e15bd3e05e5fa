// pol2.cu - total power of two recorded polarisations (Section 2: the FAST
// data record two; Eq. 1's B is the total power).
//
// With x_a = p0_a + p1_a, sum_t x_a x_b is the sum of the four
// polarisation products sum p0_a p0_b + p0_a p1_b + p1_a p0_b + p1_a p1_b,
// and sum_t x_a = sum p0_a + sum p1_a. So the exact Gram of the total power
// is a fold of the exact Gram of the 2N stacked polarisation blocks (block
// p*N + a = polarisation p of beam a), which the 8-bit Gram kernels form
// as they stand; int64 addition keeps it exact. Where the tensor-core Gram
// takes the shape it adds the polarisations itself, in pieces of 256
// samples (so its FP32 sums of products up to 255^2 stay below 2^24), and
// the pieces of a sub-integration are added here.
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

// The tensor-core route: the kernel sums the polarisations itself and
// writes the exact sums of pieces of 256 samples (interleaved by 8
// channels, [piece cell / 8][P][piece cell % 8]); a sub-integration of m
// pieces adds them up. Output interleaved the same way, or [cell][P].
__global__ void pol2_pieces_kernel(const int64_t* __restrict__ in, int64_t* __restrict__ out,
                                   int64_t n_cells, int n_chan, int P, int m, int out_public) {
  const int64_t total = n_cells * P;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total;
       o += (int64_t)gridDim.x * blockDim.x) {
    // o runs over the interleaved order: group, entry, channel in group
    const int c8 = (int)(o & 7);
    const int64_t ge = o >> 3;
    const int e = (int)(ge % P);
    const int64_t cell = (ge / P) * 8 + c8;
    const int64_t k = cell / n_chan, chan = cell - k * n_chan;
    int64_t acc = 0;
    for (int j = 0; j < m; ++j) {
      const int64_t pc = (k * m + j) * n_chan + chan;  // piece cell; pc % 8 == c8
      acc += in[((pc >> 3) * P + e) * 8 + c8];
    }
    out[out_public ? cell * P + e : o] = acc;
  }
}

}  // namespace

cudaError_t launch_pol2_pieces(const mraid_plan_s* pl, const int64_t* d_pieces, int m,
                               int64_t* d_sums, bool out_public) {
  const int64_t total = pl->n_cells * pl->psum;
  int64_t blocks = (total + 255) / 256;
  if (blocks > (int64_t)pl->sm_count * 16) blocks = (int64_t)pl->sm_count * 16;
  if (blocks < 1) return cudaSuccess;
  pol2_pieces_kernel<<<(unsigned)blocks, 256, 0, pl->stream>>>(
      d_pieces, d_sums, pl->n_cells, pl->p.n_chan, pl->psum, m, out_public ? 1 : 0);
  return cudaGetLastError();
}

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
