// Learned outflow, data and training (Sec. 3.1): capture of training rows at a
// truncation plane, the normalisation statistics of a data set, and the
// training kernel (forward pass, hand-derived backward pass, the mean squared
// error of Eq. 16, Adam).
//
// Training runs as ONE thread-block cluster.  Every CTA keeps a full copy of
// the network in shared memory and takes a contiguous slice of each batch;
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
// Weight rows and activation rows use odd strides, so a warp reading one
// column across rows hits 32 different banks.
struct TrainLayout {
  int nl = 0;
  int sizes[LBM_MLP_MAX_LAYERS + 1] = {0};
  int ws[LBM_MLP_MAX_LAYERS] = {0};      // weight row stride (odd)
  int w_off[LBM_MLP_MAX_LAYERS] = {0};   // padded W; bias follows W
  int g_off[LBM_MLP_MAX_LAYERS] = {0};   // flat (natural) parameter offsets
  int hs[LBM_MLP_MAX_LAYERS] = {0};      // activation row stride of layer inputs
  int h_off[LBM_MLP_MAX_LAYERS] = {0};
  int ds = 0;                            // delta row stride
  int chunk = 0;
  int n_params = 0;
  int w_total = 0, g0 = 0, out0 = 0, base0 = 0, ref0 = 0, d0 = 0, d1 = 0, mean0 = 0, std0 = 0;
  int loss0 = 0;                         // double slots (in floats from the start)
  int total_floats = 0;

  __host__ __device__ TrainLayout(const int* sz, int n_layers, int chunk_) {
    nl = n_layers;
    chunk = chunk_;
    int off = 0, goff = 0, maxw = 3;
    for (int l = 0; l <= nl; ++l) sizes[l] = sz[l];
    for (int l = 0; l < nl; ++l) {
      ws[l] = sizes[l] | 1;
      w_off[l] = off;
      off += sizes[l + 1] * ws[l] + sizes[l + 1];
      g_off[l] = goff;
      goff += sizes[l + 1] * sizes[l] + sizes[l + 1];
      if (sizes[l + 1] > maxw) maxw = sizes[l + 1];
    }
    n_params = goff;
    w_total = off;
    g0 = off;
    off += goff;
    for (int l = 0; l < nl; ++l) {
      hs[l] = sizes[l] | 1;
      h_off[l] = off;
      off += chunk * hs[l];
    }
    out0 = off;
    off += chunk * 3;
    base0 = off;
    off += chunk * 3;
    ref0 = off;
    off += chunk * 3;
    ds = maxw | 1;
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
    return w_off[l] + no * ws[l] + (idx - no * ni);
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

// out[s][j] = b[j] + sum_k W[j][k] h[s][k] (then the activation), for s < S,
// j < no; each thread a 4 x 4 tile (samples sg + a*nsg, units jg + b*njg).
__device__ void layer_forward(const float* __restrict__ W, int ws, const float* __restrict__ bias,
                              const float* __restrict__ h, int hs, int ni, float* out, int os,
                              int no, int S, bool hidden, int act) {
  const int njg = (no + 3) >> 2, nsg = (S + 3) >> 2;
  for (int e = threadIdx.x; e < njg * nsg; e += blockDim.x) {
    const int sg = e / njg, jg = e - sg * njg;
    int sidx[4], jidx[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      sidx[a] = min(sg + a * nsg, S - 1);
      jidx[a] = min(jg + a * njg, no - 1);
    }
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = bias[jidx[b]];
    for (int k = 0; k < ni; ++k) {
      float hv[4], wv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) hv[a] = h[sidx[a] * hs + k];
#pragma unroll
      for (int b = 0; b < 4; ++b) wv[b] = W[jidx[b] * ws + k];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(wv[b], hv[a], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int s = sg + a * nsg;
      if (s >= S) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int j = jg + b * njg;
        if (j < no) out[s * os + j] = hidden ? act_fwd(acc[a][b], act) : acc[a][b];
      }
    }
  }
}

// G[j][k] += sum_s d[s][j] h[s][k]; Gb[j] += sum_s d[s][j].
__device__ void layer_weight_grad(const float* __restrict__ d, int ds,
                                  const float* __restrict__ h, int hs, int ni, int no, int S,
                                  float* G, float* Gb) {
  const int nkg = (ni + 3) >> 2, njg = (no + 3) >> 2;
  for (int e = threadIdx.x; e < nkg * njg; e += blockDim.x) {
    const int jg = e / nkg, kg = e - jg * nkg;
    int kidx[4], jidx[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      kidx[a] = min(kg + a * nkg, ni - 1);
      jidx[a] = min(jg + a * njg, no - 1);
    }
    float acc[4][4] = {};
    for (int s = 0; s < S; ++s) {
      float dv[4], hv[4];
#pragma unroll
      for (int b = 0; b < 4; ++b) dv[b] = d[s * ds + jidx[b]];
#pragma unroll
      for (int a = 0; a < 4; ++a) hv[a] = h[s * hs + kidx[a]];
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[b][a] = fmaf(dv[b], hv[a], acc[b][a]);
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = jg + b * njg;
      if (j >= no) continue;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int k = kg + a * nkg;
        if (k < ni) G[j * ni + k] += acc[b][a];
      }
    }
  }
  for (int j = threadIdx.x; j < no; j += blockDim.x) {
    float acc = 0.f;
    for (int s = 0; s < S; ++s) acc += d[s * ds + j];
    Gb[j] += acc;
  }
}

// dn[s][k] = act'(h[s][k]) * sum_j d[s][j] W[j][k].
__device__ void layer_delta(const float* __restrict__ d, int ds, const float* __restrict__ W,
                            int ws, const float* __restrict__ h, int hs, int ni, int no, int S,
                            float* dn, int act) {
  const int nkg = (ni + 3) >> 2, nsg = (S + 3) >> 2;
  for (int e = threadIdx.x; e < nkg * nsg; e += blockDim.x) {
    const int sg = e / nkg, kg = e - sg * nkg;
    int sidx[4], kidx[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      sidx[a] = min(sg + a * nsg, S - 1);
      kidx[a] = min(kg + a * nkg, ni - 1);
    }
    float acc[4][4] = {};
    for (int j = 0; j < no; ++j) {
      float dv[4], wv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) dv[a] = d[sidx[a] * ds + j];
#pragma unroll
      for (int b = 0; b < 4; ++b) wv[b] = W[j * ws + kidx[b]];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(dv[a], wv[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int s = sg + a * nsg;
      if (s >= S) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int k = kg + b * nkg;
        if (k < ni) dn[s * ds + k] = acc[a][b] * act_grad_out(h[s * hs + k], act);
      }
    }
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
  // every CTA's copy initialised before any CTA touches another's memory
  cluster.sync();

  for (int64_t k = 0; k < p.n_steps; ++k) {
    const int64_t row0 = (int64_t)p.order[k] * B;
    for (int q = tid; q < P; q += nth) G[q] = 0.f;
    double lacc = 0.0;
    __syncthreads();
    for (int c0 = s_begin; c0 < s_end; c0 += L.chunk) {
      const int S = min(L.chunk, s_end - c0);
      // inputs (z-scored), the base values f_{3,6,7}(L-1) and the targets
      float* H0 = sm + L.h_off[0];
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
        layer_forward(Wl, L.ws[l], Wl + L.sizes[l + 1] * L.ws[l], sm + L.h_off[l], L.hs[l],
                      L.sizes[l], hidden ? sm + L.h_off[l + 1] : OUT,
                      hidden ? L.hs[l + 1] : 3, L.sizes[l + 1], S, hidden, p.act);
        __syncthreads();
      }
      // Eq. 16: r = f_{3,6,7}(L-1) + out_scale * o - f_ref; dL/do = 2 out_scale r / (3B)
      for (int e = tid; e < S * 3; e += nth) {
        const int s = e / 3, n = e - s * 3;
        const float r = BASE[e] + p.out_scale * OUT[e] - REF[e];
        lacc += (double)r * (double)r;
        Dbuf[0][s * L.ds + n] = dscale * r;
      }
      __syncthreads();
      if (p.mode != 2) {
        int cur = 0;
        for (int l = nl - 1; l >= 0; --l) {
          const int ni = L.sizes[l], no = L.sizes[l + 1];
          float* Gw = G + L.g_off[l];
          layer_weight_grad(Dbuf[cur], L.ds, sm + L.h_off[l], L.hs[l], ni, no, S, Gw,
                            Gw + no * ni);
          if (l > 0)
            layer_delta(Dbuf[cur], L.ds, W + L.w_off[l], L.ws[l], sm + L.h_off[l], L.hs[l], ni,
                        no, S, Dbuf[1 - cur], p.act);
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

    if (p.mode == 0) {
      const int64_t t = p.adam_t0 + k + 1;
      const float bc1 = (float)(1.0 - pow((double)p.beta1, (double)t));
      const float bc2 = (float)(1.0 - pow((double)p.beta2, (double)t));
      for (int q = q_begin + tid; q < q_end; q += nth) {
        float g = 0.f;
        for (int r = 0; r < C; ++r) g += cluster.map_shared_rank(G, r)[q];
        const float m = p.beta1 * p.adam_m[q] + (1.f - p.beta1) * g;
        const float v = p.beta2 * p.adam_v[q] + (1.f - p.beta2) * g * g;
        p.adam_m[q] = m;
        p.adam_v[q] = v;
        const int pq = L.padded(q);
        const float w = W[pq] - p.lr * (m / bc1) / (sqrtf(v / bc2) + p.eps);
        for (int r = 0; r < C; ++r) cluster.map_shared_rank(W, r)[pq] = w;
      }
    } else if (p.mode == 1) {
      for (int q = q_begin + tid; q < q_end; q += nth) {
        float g = 0.f;
        for (int r = 0; r < C; ++r) g += cluster.map_shared_rank(G, r)[q];
        p.grad_out[k * P + q] = g;
      }
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
  int chunk = ((batch_per_cta + 3) / 4) * 4;
  if (chunk > 128) chunk = 128;
  while (chunk > 4 && train_smem_bytes(sizes, n_layers, chunk) > smem_limit) chunk -= 4;
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
