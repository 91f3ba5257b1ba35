// East-column kernel of the NN direct-reconstruction outflow (Sec. 3.1, Eq. 15).
//
// For every node (L, y) of the east column, with L = nx - 1:
//   1. gather the 81 inputs: the nine post-stream populations of columns
//      L-1, L-2, L-3 at rows y-1, y, y+1 (periodic in y), read straight from
//      the source buffer as h_i(x - c_i) -- or, at a solid node, as the
//      reversed h_ibar(x + c_i) that bounce-back produces -- so the kernel
//      needs nothing the step kernel writes and runs after it on the same
//      buffers;
//   2. z-score them and evaluate the network (hidden tanh / LeakyReLU layers,
//      linear output) with the weights staged in shared memory;
//   3. rebuild g_i(L) = f_i(L-1) + out_scale * o_i for i = 3, 6, 7, falling
//      back to Zou & He if an output is not finite, a rebuilt population is
//      negative or the node density leaves rho_out by more than drho;
//   4. collide (BGK or MRT) and store into the destination buffer.
// The step kernel skips the east column when this kernel is active.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lattice.cuh"
#include "sim.cuh"

namespace lbm {

namespace {

constexpr int kNodes = 16;     // east nodes per block
constexpr int kThreads = 128;
constexpr int kMaxW = 81;      // widest layer input

template <typename R>
__device__ __forceinline__ R act_fn(R a, int act) {
  if (act == 0) return tanh(a);
  return a > R(0) ? a : R(0.01) * a;
}

template <typename S>
__device__ __forceinline__ double post_stream(const S* A, const NnParams& p, int x, int y, int i) {
  // post-stream, post-bounce-back population i at node (x, y), in f (not h)
  const int y_ = (y % p.ny + p.ny) % p.ny;
  const bool solid = (__ldg(p.solid_bits + (int64_t)y_ * p.words_per_row + (x >> 5)) >> (x & 31)) & 1u;
  int sx, sy, k;
  if (!solid) {
    sx = x - cx(i); sy = y_ - cy(i); k = i;
  } else {
    sx = x + cx(i); sy = y_ + cy(i); k = opp(i);
  }
  sy = (sy + p.ny) % p.ny;
  if (sx < 0) sx += p.nx;
  if (sx >= p.nx) sx -= p.nx;
  return (double)to_r<double>(A[k * p.plane + (int64_t)sy * p.pitch + sx]) + wgt<double>(k);
}

}  // namespace

template <typename S>
__global__ void __launch_bounds__(kThreads) nn_outflow_kernel(const NnParams p) {
  using R = typename Compute<S>::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);
  const R* netg = static_cast<const R*>(p.net);
  const S* __restrict__ A = static_cast<const S*>(p.src);
  S* __restrict__ B = static_cast<S*>(p.dst);

  int n_params = 0;
  for (int l = 0; l < p.n_layers; ++l) n_params += p.sizes[l] * p.sizes[l + 1] + p.sizes[l + 1];
  const int blob = n_params + 2 * 81;
  R* w = sm;                                    // weights, then in_mean, in_std
  R* act0 = w + blob;                           // [kNodes][kMaxW] ping
  R* act1 = act0 + kNodes * kMaxW;              // [kNodes][kMaxW] pong
  for (int k = threadIdx.x; k < blob; k += blockDim.x) w[k] = netg[k];

  const int L = p.nx - 1;
  const int ybase = blockIdx.x * kNodes;
  const int nn = min(kNodes, p.ny - ybase);
  __syncthreads();
  const R* in_mean = w + n_params;
  const R* in_std = in_mean + 81;
  // 1. features, z-scored
  for (int idx = threadIdx.x; idx < nn * 81; idx += blockDim.x) {
    const int n = idx / 81, f = idx % 81;
    const int k = f / 27, j = (f / 9) % 3, i = f % 9;
    const double v = post_stream(A, p, L - 1 - k, ybase + n + j - 1, i);
    act0[n * kMaxW + f] = ((R)v - in_mean[f]) / in_std[f];
  }
  __syncthreads();
  // 2. layers
  R* cur = act0;
  R* nxt = act1;
  int off = 0;
  for (int l = 0; l < p.n_layers; ++l) {
    const int n_in = p.sizes[l], n_out = p.sizes[l + 1];
    const R* W = w + off;
    const R* b = W + n_in * n_out;
    const bool last = l == p.n_layers - 1;
    for (int idx = threadIdx.x; idx < n_out * nn; idx += blockDim.x) {
      const int j = idx % n_out, n = idx / n_out;
      R acc = b[j];
      const R* wr = W + j * n_in;
      const R* xr = cur + n * kMaxW;
      for (int k = 0; k < n_in; ++k) acc = fma(wr[k], xr[k], acc);
      nxt[n * kMaxW + j] = last ? acc : act_fn<R>(acc, p.act);
    }
    off += n_in * n_out + n_out;
    __syncthreads();
    R* tmp = cur; cur = nxt; nxt = tmp;
  }
  // 3-4. one thread per node
  for (int n = threadIdx.x; n < nn; n += blockDim.x) {
    const int y = ybase + n;
    const int ym = y == 0 ? p.ny - 1 : y - 1;
    const int yp = y == p.ny - 1 ? 0 : y + 1;
    const int64_t rc = (int64_t)y * p.pitch, rm = (int64_t)ym * p.pitch, rp = (int64_t)yp * p.pitch;
    const int xm = L - 1, xp = 0;   // x = L + 1 wraps; those values are rebuilt below
    R h[9];
    h[0] = to_r<R>(A[0 * p.plane + rc + L]);
    h[1] = to_r<R>(A[1 * p.plane + rc + xm]);
    h[2] = to_r<R>(A[2 * p.plane + rm + L]);
    h[3] = to_r<R>(A[3 * p.plane + rc + xp]);
    h[4] = to_r<R>(A[4 * p.plane + rp + L]);
    h[5] = to_r<R>(A[5 * p.plane + rm + xm]);
    h[6] = to_r<R>(A[6 * p.plane + rm + xp]);
    h[7] = to_r<R>(A[7 * p.plane + rp + xp]);
    h[8] = to_r<R>(A[8 * p.plane + rp + xm]);
    const int64_t o = rc + L;
    const bool solid = (__ldg(p.solid_bits + (int64_t)y * p.words_per_row + (L >> 5)) >> (L & 31)) & 1u;
    if (solid) {
      for (int i = 0; i < 9; ++i) B[i * p.plane + o] = from_r<S>(h[opp(i)]);
      continue;
    }
    const R sc = (R)p.out_scale;
    const R s3 = sc * cur[n * kMaxW + 0];
    const R s6 = sc * cur[n * kMaxW + 1];
    const R s7 = sc * cur[n * kMaxW + 2];
    // bases of Eq. 15: post-stream h_i(L-1, y)
    const R b3 = (R)(post_stream(A, p, L - 1, y, 3) - wgt<double>(3));
    const R b6 = (R)(post_stream(A, p, L - 1, y, 6) - wgt<double>(6));
    const R b7 = (R)(post_stream(A, p, L - 1, y, 7) - wgt<double>(7));
    R hn[9];
    for (int i = 0; i < 9; ++i) hn[i] = h[i];
    hn[3] = b3 + s3;
    hn[6] = b6 + s6;
    hn[7] = b7 + s7;
    R drho_n, jx_n, jy_n;
    moments_shifted(hn, drho_n, jx_n, jy_n);
    (void)jx_n; (void)jy_n;
    bool ok = isfinite((double)s3) && isfinite((double)s6) && isfinite((double)s7);
    ok = ok && (hn[3] + wgt<R>(3) >= R(0)) && (hn[6] + wgt<R>(6) >= R(0)) &&
         (hn[7] + wgt<R>(7) >= R(0));
    ok = ok && (fabs((double)((R(1) + drho_n) - (R)p.rho_out)) <= p.fallback_drho);
    if (ok) {
      for (int i = 0; i < 9; ++i) h[i] = hn[i];
    } else {
      zouhe_east<R>(h, (R)p.rho_out);
      atomicAdd(p.fallbacks, 1ull);
    }
    R drho, ux, uy;
    if (p.collision == LBM_BGK) {
      collide_bgk<R>(h, (R)p.omega, drho, ux, uy);
    } else {
      MrtRates<R> mrt{(R)p.mrt_se, (R)p.mrt_seps, (R)p.mrt_sq, (R)p.mrt_snu};
      collide_mrt<R>(h, mrt, drho, ux, uy);
    }
    if (!(fabs((double)drho) < 1e30)) atomicOr(p.status, DEV_NONFINITE);
    for (int i = 0; i < 9; ++i) B[i * p.plane + o] = from_r<S>(h[i]);
  }
}

template <typename S>
static void launch_nn_t(const NnParams& p, cudaStream_t s) {
  using R = typename Compute<S>::R;
  int n_params = 0;
  for (int l = 0; l < p.n_layers; ++l) n_params += p.sizes[l] * p.sizes[l + 1] + p.sizes[l + 1];
  const size_t smem = sizeof(R) * ((size_t)n_params + 2 * 81 + 2 * kNodes * kMaxW);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(nn_outflow_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    attr_set = true;
  }
  const int blocks = (p.ny + kNodes - 1) / kNodes;
  nn_outflow_kernel<S><<<blocks, kThreads, smem, s>>>(p);
}

void launch_nn_outflow(int prec, const NnParams& p, cudaStream_t s) {
  if (prec == LBM_FP64) launch_nn_t<double>(p, s);
  else if (prec == LBM_FP32) launch_nn_t<float>(p, s);
  else launch_nn_t<__half>(p, s);
}

}  // namespace lbm
