// Learned outflow, data and training (Sec. 3.1): capture of training rows at a
// truncation plane, the normalisation statistics of a data set, and the
// training kernel (forward pass, hand-derived backward pass, the mean squared
// error of Eq. 16, Adam).
//
// Training runs as ONE thread-block cluster.  Every CTA keeps a full copy of
// the network in shared memory and takes a contiguous slice of each batch;
// the forward products, the backward deltas and the weight gradients of a
// slice run on the tensor cores (mma.sync on TF32 operands split into high
// and low parts, 3xTF32, FP32 accumulation: FP32-level products);
// the per-CTA gradients are summed in a fixed CTA order through distributed
// shared memory by the CTA that owns each parameter, which applies Adam and
// writes the new value into every CTA's copy.  Two cluster barriers per Adam
// step; all steps of a call run in one launch.  Sums have a fixed order, so a
// run is bitwise reproducible for a given cluster size.
#include <cooperative_groups.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "../../include/lbm.h"
#include "lattice.cuh"
#include "mma_tf32.cuh"
#include "sim.cuh"

namespace cg = cooperative_groups;

namespace lbm {

// ---- capture of training rows ---------------------------------------------

__device__ __forceinline__ double pop_value(const double* a, int64_t k) { return a[k]; }
__device__ __forceinline__ double pop_value(const float* a, int64_t k) { return a[k]; }
__device__ __forceinline__ double pop_value(const __half* a, int64_t k) {
  return __half2float(a[k]);
}

// One thread per lattice row y: the post-stream populations (pull from the
// post-collision state A, a solid node reversing what arrives, Eq. 11) of
// columns x_t-1..x_t-3, rows y-1..y+1 (81 inputs of Eq. 15, index
// k*27 + j*9 + i), then f_3, f_6, f_7 at (x_t, y).
template <typename S>
__device__ __forceinline__ void capture_row(const CaptureParams& p, int x_t, int y, float* out) {
  const S* __restrict__ A = static_cast<const S*>(p.src);
  auto post = [&](int i, int x, int yy) -> float {
    yy = yy < 0 ? yy + p.ny : (yy >= p.ny ? yy - p.ny : yy);
    const uint32_t word = p.solid_bits[(int64_t)yy * p.words_per_row + (x >> 5)];
    if ((word >> (x & 31)) & 1u) i = opp(i);
    int sy = yy - cy(i);
    sy = sy < 0 ? sy + p.ny : (sy >= p.ny ? sy - p.ny : sy);
    const int sx = x - cx(i);
    return (float)(pop_value(A, (int64_t)i * p.plane + (int64_t)sy * p.pitch + sx) + wgt<double>(i));
  };
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 3; ++j)
      for (int i = 0; i < 9; ++i) out[k * 27 + j * 9 + i] = post(i, x_t - 1 - k, y - 1 + j);
  out[81] = post(3, x_t, y);
  out[82] = post(6, x_t, y);
  out[83] = post(7, x_t, y);
}

template <typename S>
__global__ void capture_kernel(const CaptureParams p) {
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= p.ny) return;
  capture_row<S>(p, p.x_t, y, p.out + (int64_t)y * kRowFloats);
}

// Snapshot (Sec. 3.1: the training set is one converged snapshot, each
// column a batch): column x_t + blockIdx.y, rows in order, one batch of ny
// rows per column.
template <typename S>
__global__ void snapshot_kernel(const CaptureParams p) {
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= p.ny) return;
  const int c = blockIdx.y;
  capture_row<S>(p, p.x_t + c, y, p.out + ((int64_t)c * p.ny + y) * kRowFloats);
}

void launch_capture(int prec, const CaptureParams& p, cudaStream_t s) {
  const int grid = (p.ny + 127) / 128;
  if (prec == LBM_FP64) capture_kernel<double><<<grid, 128, 0, s>>>(p);
  else if (prec == LBM_FP32) capture_kernel<float><<<grid, 128, 0, s>>>(p);
  else capture_kernel<__half><<<grid, 128, 0, s>>>(p);
}

void launch_snapshot(int prec, const CaptureParams& p, int n_cols, cudaStream_t s) {
  const dim3 grid((unsigned)((p.ny + 127) / 128), (unsigned)n_cols);
  if (prec == LBM_FP64) snapshot_kernel<double><<<grid, 128, 0, s>>>(p);
  else if (prec == LBM_FP32) snapshot_kernel<float><<<grid, 128, 0, s>>>(p);
  else snapshot_kernel<__half><<<grid, 128, 0, s>>>(p);
}

// ---- data-set statistics ------------------------------------------------------
// Column c < 81: input feature c.  Columns 81..83: the residual targets
// f_ref,n - f_{3,6,7}(L-1) (inputs 12, 15, 16), pooled over n for out_scale.
constexpr int kStatCols = 84;
constexpr int kStatBlocks = 512;

__device__ __forceinline__ double stat_value(const float* r, int c) {
  if (c < 81) return r[c];
  const int base = c == 81 ? 12 : (c == 82 ? 15 : 16);
  return (double)r[c] - (double)r[base];
}

// pass 0: per-block sums of each column; pass 1: sums of squared deviations
// from mean[] (columns >= 81 all use the pooled residual mean mean[81]).
__global__ void stats_partial_kernel(const float* __restrict__ rows, int64_t n, int pass,
                                     const double* __restrict__ mean, double* partial) {
  const int c = threadIdx.x;
  if (c >= kStatCols) return;
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per;
  const int64_t r1 = r0 + per < n ? r0 + per : n;
  const double m = pass == 0 ? 0.0 : mean[c < 81 ? c : 81];
  double acc = 0.0;
  for (int64_t r = r0; r < r1; ++r) {
    const double v = stat_value(rows + r * kRowFloats, c);
    acc += pass == 0 ? v : (v - m) * (v - m);
  }
  partial[(int64_t)blockIdx.x * kStatCols + c] = acc;
}

// Sum the block partials in block order.  pass 0 -> mean[c]; the residual
// columns are pooled into mean[81].  pass 1 -> var[c] likewise.
__global__ void stats_reduce_kernel(const double* __restrict__ partial, int blocks, int64_t n,
                                    double* out) {
  __shared__ double col[kStatCols];
  const int c = threadIdx.x;
  if (c < kStatCols) {
    double acc = 0.0;
    for (int b = 0; b < blocks; ++b) acc += partial[(int64_t)b * kStatCols + c];
    col[c] = acc;
  }
  __syncthreads();
  if (c < 81) out[c] = col[c] / (double)n;
  if (c == 81) out[81] = (col[81] + col[82] + col[83]) / (3.0 * (double)n);
}

void dataset_stats(const float* rows, int64_t n, double* scratch, cudaStream_t s) {
  // scratch: partial[kStatBlocks * 84] | mean[82] | var[82]
  double* partial = scratch;
  double* mean = scratch + (int64_t)kStatBlocks * kStatCols;
  double* var = mean + 82;
  const int blocks = (int)std::min<int64_t>(kStatBlocks, std::max<int64_t>(1, n));
  stats_partial_kernel<<<blocks, 96, 0, s>>>(rows, n, 0, mean, partial);
  stats_reduce_kernel<<<1, 96, 0, s>>>(partial, blocks, n, mean);
  stats_partial_kernel<<<blocks, 96, 0, s>>>(rows, n, 1, mean, partial);
  stats_reduce_kernel<<<1, 96, 0, s>>>(partial, blocks, n, var);
}

int dataset_stats_scratch_doubles() { return kStatBlocks * kStatCols + 2 * 82; }

// ---- training ---------------------------------------------------------------

// Shared-memory layout of the training kernel, identical on host and device.
// The layer products run on the tensor cores (3xTF32 mma.sync), so every
// operand is zero-padded: a layer's inputs to a multiple of 8 columns (kp),
// its outputs to a multiple of 8 (np8), samples of a chunk to a multiple of
// 16.  Row strides are 4 more than a multiple of 8, which spreads the rows of
// a fragment load over distinct banks.
struct TrainLayout {
  int nl = 0;
  int sizes[LBM_MLP_MAX_LAYERS + 1] = {0};
  int kp[LBM_MLP_MAX_LAYERS] = {0};      // inputs of layer l padded to a multiple of 8
  int np8[LBM_MLP_MAX_LAYERS] = {0};     // outputs of layer l padded to a multiple of 8
  int ws[LBM_MLP_MAX_LAYERS] = {0};      // weight row stride (kp + 4)
  int w_off[LBM_MLP_MAX_LAYERS] = {0};   // W [np8][ws]; bias [no] follows
  int g_off[LBM_MLP_MAX_LAYERS] = {0};   // flat (natural) parameter offsets
  int hs[LBM_MLP_MAX_LAYERS] = {0};      // activation row stride of layer inputs (kp + 4)
  int h_off[LBM_MLP_MAX_LAYERS] = {0};
  int os = 0;                            // output row stride (np8 of the last layer + 4)
  int ds = 0;                            // delta row stride
  int chunk = 0;                         // samples per chunk (a multiple of 16)
  int n_params = 0;
  int w_total = 0, g0 = 0, out0 = 0, base0 = 0, ref0 = 0, d0 = 0, d1 = 0, mean0 = 0, std0 = 0;
  int loss0 = 0;                         // double slots (in floats from the start)
  int total_floats = 0;

  __host__ __device__ TrainLayout(const int* sz, int n_layers, int chunk_) {
    nl = n_layers;
    chunk = chunk_;
    int off = 0, goff = 0, maxd = 8;
    for (int l = 0; l <= nl; ++l) sizes[l] = sz[l];
    for (int l = 0; l < nl; ++l) {
      kp[l] = (sizes[l] + 7) / 8 * 8;
      np8[l] = (sizes[l + 1] + 7) / 8 * 8;
      ws[l] = kp[l] + 4;
      w_off[l] = off;
      off += np8[l] * ws[l] + sizes[l + 1];
      g_off[l] = goff;
      goff += sizes[l + 1] * sizes[l] + sizes[l + 1];
      const int m16 = (sizes[l + 1] + 15) / 16 * 16;   // rows of a weight-gradient product
      if (m16 > maxd) maxd = m16;
      if (kp[l] > maxd) maxd = kp[l];
    }
    n_params = goff;
    w_total = off;
    g0 = off;
    off += goff;
    for (int l = 0; l < nl; ++l) {
      hs[l] = kp[l] + 4;
      h_off[l] = off;
      off += chunk * hs[l];
    }
    os = np8[nl - 1] + 4;
    out0 = off;
    off += chunk * os;
    base0 = off;
    off += chunk * 3;
    ref0 = off;
    off += chunk * 3;
    ds = maxd + 4;
    d0 = off;
    off += chunk * ds;
    d1 = off;
    off += chunk * ds;
    mean0 = off;
    off += 81;
    std0 = off;
    off += 81;
    off = (off + 1) & ~1;   // 8-byte alignment for the doubles
    loss0 = off;
    off += 2 * 40;          // 32 warp partials + total, as doubles
    total_floats = off;
  }

  // padded shared-memory index of flat parameter q
  __host__ __device__ int padded(int q) const {
    int l = 0;
    while (l + 1 < nl && q >= g_off[l + 1]) ++l;
    const int idx = q - g_off[l];
    const int ni = sizes[l], no = sizes[l + 1];
    if (idx < no * ni) {
      const int j = idx / ni;
      return w_off[l] + j * ws[l] + (idx - j * ni);
    }
    return w_off[l] + np8[l] * ws[l] + (idx - no * ni);
  }
};

constexpr int kTrainThreads = 512;

__device__ __forceinline__ float act_fwd(float a, int act) {
  if (act == 0) return tanhf(a);
  return a > 0.f ? a : 0.01f * a;
}

// derivative of the activation from its output h (tanh' = 1 - h^2; the
// LeakyReLU output is positive exactly when its input is)
__device__ __forceinline__ float act_grad_out(float h, int act) {
  if (act == 0) return 1.f - h * h;
  return h > 0.f ? 1.f : 0.01f;
}

// One 16 x 8 tile (rows m0.., columns n0..) of sum_k A(m, k) B(k, n) over
// k < K (a multiple of 8) into c, on the tensor cores with 3xTF32 (the two
// small cross terms first).  a(m, k) and b(k, n) read shared memory.
template <typename FA, typename FB>
__device__ __forceinline__ void tile_3xtf32(float c[4], int m0, int n0, int K, FA a, FB b) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int k0 = 0; k0 < K; k0 += 8) {
    uint32_t ah[4], al[4], bh0, bl0, bh1, bl1;
    tf32_split(a(m0 + g, k0 + t), ah[0], al[0]);
    tf32_split(a(m0 + g + 8, k0 + t), ah[1], al[1]);
    tf32_split(a(m0 + g, k0 + t + 4), ah[2], al[2]);
    tf32_split(a(m0 + g + 8, k0 + t + 4), ah[3], al[3]);
    tf32_split(b(k0 + t, n0 + g), bh0, bl0);
    tf32_split(b(k0 + t + 4, n0 + g), bh1, bl1);
    mma_tf32_1688(c, al, bh0, bh1);
    mma_tf32_1688(c, ah, bl0, bl1);
    mma_tf32_1688(c, ah, bh0, bh1);
  }
}

// out[s][j] = act(b[j] + sum_k W[j][k] h[s][k]) for s < M (a multiple of 16)
// and j < no8 (the padded outputs come out zero: zero weights and bias, and
// act(0) = 0).  The warps take the 16 x 8 tiles in turn.
__device__ void layer_forward(const float* W, int ws, const float* bias, const float* h, int hs,
                              int kp, float* out, int os, int no, int no8, int M, bool hidden,
                              int act) {
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int nt = no8 / 8, tiles = (M / 16) * nt;
  for (int e = warp; e < tiles; e += nw) {
    const int m0 = (e / nt) * 16, n0 = (e % nt) * 8;
    const int j0 = n0 + 2 * t, j1 = j0 + 1;
    const float b0 = j0 < no ? bias[j0] : 0.f, b1 = j1 < no ? bias[j1] : 0.f;
    float c[4] = {b0, b1, b0, b1};
    tile_3xtf32(c, m0, n0, kp, [&](int m, int k) { return h[m * hs + k]; },
                [&](int k, int n) { return W[n * ws + k]; });
    float* o0 = out + (m0 + g) * os + j0;
    float* o1 = out + (m0 + g + 8) * os + j0;
    o0[0] = hidden ? act_fwd(c[0], act) : c[0];
    o0[1] = hidden ? act_fwd(c[1], act) : c[1];
    o1[0] = hidden ? act_fwd(c[2], act) : c[2];
    o1[1] = hidden ? act_fwd(c[3], act) : c[3];
  }
}

// G[j][k] += sum_{s < K} d[s][j] h[s][k] (j < no, k < ni; K a multiple of 8,
// rows of d beyond the chunk's samples zero) and Gb[j] += sum_s d[s][j].
__device__ void layer_weight_grad(const float* d, int ds, const float* h, int hs, int ni, int kp,
                                  int no, int K, float* G, float* Gb) {
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int nt = kp / 8, tiles = ((no + 15) / 16) * nt;
  for (int e = warp; e < tiles; e += nw) {
    const int m0 = (e / nt) * 16, n0 = (e % nt) * 8;
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    tile_3xtf32(c, m0, n0, K, [&](int m, int k) { return d[k * ds + m]; },
                [&](int k, int n) { return h[k * hs + n]; });
    const int ja = m0 + g, jb = ja + 8, k0 = n0 + 2 * t;
    if (ja < no) {
      if (k0 < ni) G[ja * ni + k0] += c[0];
      if (k0 + 1 < ni) G[ja * ni + k0 + 1] += c[1];
    }
    if (jb < no) {
      if (k0 < ni) G[jb * ni + k0] += c[2];
      if (k0 + 1 < ni) G[jb * ni + k0 + 1] += c[3];
    }
  }
  for (int j = threadIdx.x; j < no; j += blockDim.x) {
    float acc = 0.f;
    for (int s = 0; s < K; ++s) acc += d[s * ds + j];
    Gb[j] += acc;
  }
}

// dn[s][k] = act'(h[s][k]) * sum_{j < no8} d[s][j] W[j][k] for s < M, k < kp.
__device__ void layer_delta(const float* d, int ds, const float* W, int ws, const float* h,
                            int hs, int kp, int no8, int M, float* dn, int act) {
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int nt = kp / 8, tiles = (M / 16) * nt;
  for (int e = warp; e < tiles; e += nw) {
    const int m0 = (e / nt) * 16, n0 = (e % nt) * 8;
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    tile_3xtf32(c, m0, n0, no8, [&](int m, int k) { return d[m * ds + k]; },
                [&](int k, int n) { return W[k * ws + n]; });
    const int sa = m0 + g, sb = sa + 8, k0 = n0 + 2 * t;
    dn[sa * ds + k0] = c[0] * act_grad_out(h[sa * hs + k0], act);
    dn[sa * ds + k0 + 1] = c[1] * act_grad_out(h[sa * hs + k0 + 1], act);
    dn[sb * ds + k0] = c[2] * act_grad_out(h[sb * hs + k0], act);
    dn[sb * ds + k0 + 1] = c[3] * act_grad_out(h[sb * hs + k0 + 1], act);
  }
}

__global__ void __launch_bounds__(kTrainThreads, 1) nn_train_kernel(const TrainParams p) {
  extern __shared__ __align__(16) float sm[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int C = (int)cluster.num_blocks();
  const int tid = threadIdx.x, nth = blockDim.x;
  const TrainLayout L(p.sizes, p.n_layers, p.chunk);
  const int P = L.n_params, nl = L.nl;
  float* W = sm;
  float* G = sm + L.g0;
  float* OUT = sm + L.out0;
  float* BASE = sm + L.base0;
  float* REF = sm + L.ref0;
  float* Dbuf[2] = {sm + L.d0, sm + L.d1};
  float* MEAN = sm + L.mean0;
  float* STD = sm + L.std0;
  double* LOSS = reinterpret_cast<double*>(sm + L.loss0);

  // weights with zero padding (the padded rows and columns stay zero: Adam
  // writes only real parameters)
  for (int q = tid; q < L.w_total; q += nth) W[q] = 0.f;
  __syncthreads();
  for (int q = tid; q < P; q += nth) W[L.padded(q)] = p.params[q];
  for (int c = tid; c < 81; c += nth) {
    MEAN[c] = p.in_mean[c];
    STD[c] = p.in_std[c];
  }
  const int B = p.batch_rows;
  const int per = (B + C - 1) / C;
  const int s_begin = min(B, rank * per), s_end = min(B, s_begin + per);
  const int pc = (P + C - 1) / C;
  const int q_begin = min(P, rank * pc), q_end = min(P, q_begin + pc);
  const float dscale = 2.f * p.out_scale / (3.f * (float)B);
  // beta^t of the first step of this launch (t = adam_t0 + 1), then one
  // multiplication per step
  double b1t = pow((double)p.beta1, (double)(p.adam_t0 + 1));
  double b2t = pow((double)p.beta2, (double)(p.adam_t0 + 1));
  // every CTA's copy initialised before any CTA touches another's memory
  cluster.sync();

  for (int64_t k = 0; k < p.n_steps; ++k) {
    const int64_t row0 = (int64_t)p.order[k] * B;
    for (int q = tid; q < P; q += nth) G[q] = 0.f;
    double lacc = 0.0;
    __syncthreads();
    for (int c0 = s_begin; c0 < s_end; c0 += L.chunk) {
      const int S = min(L.chunk, s_end - c0);
      const int M = (S + 15) / 16 * 16;     // rows of the forward and delta products
      const int K8 = (S + 7) / 8 * 8;       // samples summed by the weight gradients
      // inputs (z-scored; padding zero), the base values f_{3,6,7}(L-1), the
      // targets, and a zero output delta (its padding is read as zero)
      float* H0 = sm + L.h_off[0];
      for (int e = tid; e < M * L.kp[0]; e += nth) {
        const int s = e / L.kp[0], c = e - s * L.kp[0];
        H0[s * L.hs[0] + c] = 0.f;
      }
      for (int e = tid; e < M * L.ds; e += nth) Dbuf[0][e] = 0.f;
      __syncthreads();
      for (int e = tid; e < S * kRowFloats; e += nth) {
        const int s = e / kRowFloats, c = e - s * kRowFloats;
        const float v = p.rows[(row0 + c0 + s) * kRowFloats + c];
        if (c < 81) H0[s * L.hs[0] + c] = (v - MEAN[c]) / STD[c];
        else REF[s * 3 + (c - 81)] = v;
        if (c == 12) BASE[s * 3 + 0] = v;
        else if (c == 15) BASE[s * 3 + 1] = v;
        else if (c == 16) BASE[s * 3 + 2] = v;
      }
      __syncthreads();
      for (int l = 0; l < nl; ++l) {
        const bool hidden = l < nl - 1;
        const float* Wl = W + L.w_off[l];
        layer_forward(Wl, L.ws[l], Wl + L.np8[l] * L.ws[l], sm + L.h_off[l], L.hs[l], L.kp[l],
                      hidden ? sm + L.h_off[l + 1] : OUT, hidden ? L.hs[l + 1] : L.os,
                      L.sizes[l + 1], L.np8[l], M, hidden, p.act);
        __syncthreads();
      }
      // Eq. 16: r = f_{3,6,7}(L-1) + out_scale * o - f_ref; dL/do = 2 out_scale r / (3B)
      for (int e = tid; e < S * 3; e += nth) {
        const int s = e / 3, n = e - s * 3;
        const float r = BASE[e] + p.out_scale * OUT[s * L.os + n] - REF[e];
        lacc += (double)r * (double)r;
        Dbuf[0][s * L.ds + n] = dscale * r;
      }
      __syncthreads();
      if (p.mode != 2) {
        int cur = 0;
        for (int l = nl - 1; l >= 0; --l) {
          const int ni = L.sizes[l], no = L.sizes[l + 1];
          float* Gw = G + L.g_off[l];
          layer_weight_grad(Dbuf[cur], L.ds, sm + L.h_off[l], L.hs[l], ni, L.kp[l], no, K8, Gw,
                            Gw + no * ni);
          if (l > 0)
            layer_delta(Dbuf[cur], L.ds, W + L.w_off[l], L.ws[l], sm + L.h_off[l], L.hs[l],
                        L.kp[l], L.np8[l], M, Dbuf[1 - cur], p.act);
          __syncthreads();
          cur = 1 - cur;
        }
      }
    }
    // block sum of the squared residuals, in warp order
    for (int o = 16; o > 0; o >>= 1) lacc += __shfl_down_sync(0xffffffffu, lacc, o);
    if ((tid & 31) == 0) LOSS[tid >> 5] = lacc;
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0;
      for (int w = 0; w < nth / 32; ++w) tot += LOSS[w];
      LOSS[32] = tot;
    }
    cluster.sync();   // every CTA's G and loss are complete

    // the cluster's gradient of parameter q: the CTAs' partial sums added in
    // CTA order (all remote loads issued before the first addition)
    auto cluster_grad = [&](int q) {
      float gv[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) gv[r] = r < C ? cluster.map_shared_rank(G, r)[q] : 0.f;
      float g = 0.f;
#pragma unroll
      for (int r = 0; r < 16; ++r)
        if (r < C) g += gv[r];
      return g;
    };
    if (p.mode == 0) {
      // bias corrections 1 - beta^t, t = adam_t0 + k + 1, from the running powers
      const float bc1 = (float)(1.0 - b1t), bc2 = (float)(1.0 - b2t);
      for (int q = q_begin + tid; q < q_end; q += nth) {
        const float g = cluster_grad(q);
        const float m = p.beta1 * p.adam_m[q] + (1.f - p.beta1) * g;
        const float v = p.beta2 * p.adam_v[q] + (1.f - p.beta2) * g * g;
        p.adam_m[q] = m;
        p.adam_v[q] = v;
        const int pq = L.padded(q);
        const float w = W[pq] - p.lr * (m / bc1) / (sqrtf(v / bc2) + p.eps);
        for (int r = 0; r < C; ++r) cluster.map_shared_rank(W, r)[pq] = w;
      }
      b1t *= (double)p.beta1;
      b2t *= (double)p.beta2;
    } else if (p.mode == 1) {
      for (int q = q_begin + tid; q < q_end; q += nth) p.grad_out[k * P + q] = cluster_grad(q);
    }
    if (rank == 0 && tid == 0) {
      double tot = 0.0;
      for (int r = 0; r < C; ++r) tot += cluster.map_shared_rank(LOSS, r)[32];
      p.loss_log[k] = tot / (3.0 * (double)B);
    }
    cluster.sync();   // new weights everywhere; G and LOSS free for reuse
  }
  if (p.mode == 0)
    for (int q = q_begin + tid; q < q_end; q += nth) p.params[q] = W[L.padded(q)];
}

int train_smem_bytes(const int* sizes, int n_layers, int chunk) {
  return TrainLayout(sizes, n_layers, chunk).total_floats * (int)sizeof(float);
}

int train_max_chunk(const int* sizes, int n_layers, int batch_per_cta, int smem_limit) {
  // a multiple of 16 samples (the rows of a tensor-core tile)
  int chunk = ((batch_per_cta + 15) / 16) * 16;
  if (chunk > 128) chunk = 128;
  while (chunk > 16 && train_smem_bytes(sizes, n_layers, chunk) > smem_limit) chunk -= 16;
  return train_smem_bytes(sizes, n_layers, chunk) <= smem_limit ? chunk : 0;
}

cudaError_t launch_train(const TrainParams& p, int cluster, cudaStream_t s) {
  const int smem = train_smem_bytes(p.sizes, p.n_layers, p.chunk);
  cudaError_t e = cudaFuncSetAttribute(nn_train_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (cluster > 8) {
    e = cudaFuncSetAttribute(nn_train_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)cluster);
  cfg.blockDim = dim3(kTrainThreads);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, nn_train_kernel, p);
}

// Largest cluster size in {16, 8, 4, 2, 1} (not above max_cluster) that the
// device can place with this shared-memory footprint.
int train_cluster_size(const TrainParams& p, int max_cluster) {
  const int smem = train_smem_bytes(p.sizes, p.n_layers, p.chunk);
  if (cudaFuncSetAttribute(nn_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
      cudaSuccess)
    return 0;
  for (int c = 16; c >= 1; c >>= 1) {
    if (c > max_cluster) continue;
    if (c > 8 && cudaFuncSetAttribute(nn_train_kernel,
                                      cudaFuncAttributeNonPortableClusterSizeAllowed,
                                      1) != cudaSuccess)
      continue;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)c);
    cfg.blockDim = dim3(kTrainThreads);
    cfg.dynamicSmemBytes = (size_t)smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, nn_train_kernel, &cfg) == cudaSuccess && n > 0)
      return c;
    cudaGetLastError();
  }
  return 0;
}

}  // namespace lbm
