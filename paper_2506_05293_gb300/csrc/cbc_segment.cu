// Training of the CBC tuner through short simulation segments (Sec. 4.2 and
// its tuning-procedure figure): forward segments on east strips, their loss,
// the reverse (adjoint) pass and Adam, all in FP64 on the device.
//
// A segment starts from a reference state of the truncated lattice, runs n_t
// steps with the characteristic outflow (Eqs. 17-28) whose sigma (and kappa2)
// the tuner predicts per east node, and is compared with the reference at the
// same time over the last n_t columns:
//   loss = mean(rho - rho_ref)^2 + mean over both components (U - U_ref)^2.
// The loss region at t0 + n_t depends only on the last 2 n_t columns at t0
// (one column per step of pull streaming; the east node's stencil reaches two
// columns back), so every segment lives on a strip of W = max(2 n_t, 3) east
// columns; the strip's west edge pulls a frozen value, which never reaches the
// loss region nor the adjoint's support.
//
// Reverse pass, step t+1 -> t, given lambda_{t+1} = dL/df(t+1):
//  * interior node: f(t+1) = BGK(p), p_i = f_i(x - c_i, t); mu = J_BGK(p)^T lambda
//    in closed form (the equilibrium's derivatives in rho, u, v);
//  * east node: its inputs are the moments (rho, u, v) of the five stencil
//    nodes whose differences give the derivatives, the six known pulled
//    populations, and sigma and kappa2, which the tuner computes from the
//    derivatives.  One warp per east node: forward-mode (dual number)
//    evaluations of the same templated functions the forward pass runs give
//    the tuner's Jacobian (one lane per feature) and the 23 directional
//    derivatives of lambda . node (one lane per input); the moments' adjoints
//    add the path through the tuner and become population adjoints;
//  * lambda_t gathers, per population, the consumers' mu and the east nodes'
//    input adjoints (a fixed order: bitwise reproducible).
// The sensitivities to sigma and kappa2 of every east node and step, with the
// tuner's features, are records; the parameter gradient backpropagates every
// record through the tuner and sums them per block and then over blocks in a
// fixed order.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lattice.cuh"
#include "sim.cuh"

namespace lbm {
namespace {

constexpr int kEastInputs = 51;           // 5 stencil nodes x 9 + 6 known pulls
constexpr int kSegMaxW = 32;              // widest hidden layer of the tuner
constexpr int kRecWidth = 8;              // features (6), dL/dsigma, dL/dkappa2
constexpr int kGradThreads = 128;
constexpr int kGradChunk = 64;            // records per chunk of the gradient kernel
constexpr int kGradBlocks = 152;

// ---- forward-mode dual numbers ------------------------------------------
struct Dual {
  double v, d;
};
__device__ __forceinline__ Dual mk(double v) { return {v, 0.0}; }
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const double q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ Dual operator+(Dual a, double b) { return {a.v + b, a.d}; }
__device__ __forceinline__ Dual operator+(double a, Dual b) { return {a + b.v, b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, double b) { return {a.v - b, a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, double b) { return {a.v * b, a.d * b}; }
__device__ __forceinline__ Dual operator*(double a, Dual b) { return {a * b.v, a * b.d}; }
__device__ __forceinline__ Dual operator/(Dual a, double b) { return {a.v / b, a.d / b}; }

template <typename T> __device__ __forceinline__ T mk_t(double v);
template <> __device__ __forceinline__ double mk_t<double>(double v) { return v; }
template <> __device__ __forceinline__ Dual mk_t<Dual>(double v) { return mk(v); }

__device__ __forceinline__ double value(double a) { return a; }
__device__ __forceinline__ double value(Dual a) { return a.v; }
__device__ __forceinline__ double tanh_g(double a) { return tanh(a); }
__device__ __forceinline__ Dual tanh_g(Dual a) {
  const double t = tanh(a.v);
  return {t, (1.0 - t * t) * a.d};
}
__device__ __forceinline__ double sigmoid_g(double a) { return 1.0 / (1.0 + exp(-a)); }
__device__ __forceinline__ Dual sigmoid_g(Dual a) {
  const double s = 1.0 / (1.0 + exp(-a.v));
  return {s, s * (1.0 - s) * a.d};
}
template <typename T>
__device__ __forceinline__ T act_g(T a, int act) {
  if (act == 0) return tanh_g(a);
  return value(a) > 0.0 ? a : a * 0.01;     // LeakyReLU, slope 0.01
}

struct SegParams {
  int n_seg, ny, W, n_t, bank_w;
  double omega, rho_out, sig_max, kap, kfac;
  int exact;
  // tuner: per layer W (n_out x n_in, row-major) then b; z-scored inputs
  int n_layers, sizes[LBM_MLP_MAX_LAYERS + 1], act;
  const double* net;
  const double* in_mean;
  const double* in_std;
  int64_t n_params;
  // data
  const double* bank;     // [n_states][9][ny][bank_w]
  const int* init_idx;    // [n_seg]
  const int* final_idx;   // [n_seg]
  double* hist;           // [n_seg][n_t + 1][9][ny][W]
  double* lam_in;         // [n_seg][9][ny][W]   lambda_{t+1}
  double* lam_out;        // [n_seg][9][ny][W]   lambda_t
  double* mu;             // [n_seg][9][ny][W]
  double* east;           // [n_seg][ny][kEastInputs]
  double* rec;            // [n_seg][n_t][ny][kRecWidth]
  double* loss_part;      // per block of the loss kernel
};

__device__ __forceinline__ int64_t node_plane(const SegParams& p) { return (int64_t)p.ny * p.W; }
__device__ __forceinline__ double* hist_at(const SegParams& p, int s, int t) {
  return p.hist + ((int64_t)s * (p.n_t + 1) + t) * 9 * node_plane(p);
}
__device__ __forceinline__ int wrap(int y, int ny) { return y < 0 ? y + ny : (y >= ny ? y - ny : y); }

template <typename T>
__device__ __forceinline__ void moments_g(const T f[9], T& rho, T& u, T& v) {
  rho = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
  const T jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
  const T jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
  u = jx / rho;
  v = jy / rho;
}

// Eq. 3 with c_s^2 = 1/3
template <typename T>
__device__ __forceinline__ void feq_g(T rho, T u, T v, T out[9]) {
  const T usq = u * u + v * v;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const T cu = (double)cx(i) * u + (double)cy(i) * v;
    out[i] = wgt<double>(i) * rho * (1.0 + 3.0 * cu + 4.5 * (cu * cu) - 1.5 * usq);
  }
}

// Eq. 2
template <typename T>
__device__ __forceinline__ void bgk_g(const T g[9], double omega, T out[9]) {
  T rho, u, v, fe[9];
  moments_g(g, rho, u, v);
  feq_g(rho, u, v, fe);
#pragma unroll
  for (int i = 0; i < 9; ++i) out[i] = g[i] - omega * (g[i] - fe[i]);
}

template <typename T>
__device__ void tuner_g(const SegParams& p, const T x[6], T s[2]) {
  T a[kSegMaxW], b[kSegMaxW];
  for (int k = 0; k < 6; ++k) a[k] = (x[k] - p.in_mean[k]) / p.in_std[k];
  int64_t off = 0;
  for (int l = 0; l < p.n_layers; ++l) {
    const int n_in = p.sizes[l], n_out = p.sizes[l + 1];
    const double* Wl = p.net + off;
    const double* bl = Wl + (int64_t)n_in * n_out;
    const bool last = l == p.n_layers - 1;
    for (int j = 0; j < n_out; ++j) {
      T acc = mk_t<T>(bl[j]);
      for (int k = 0; k < n_in; ++k) acc = acc + Wl[j * n_in + k] * a[k];
      b[j] = last ? acc : act_g(acc, p.act);
    }
    for (int j = 0; j < n_out; ++j) a[j] = b[j];
    off += (int64_t)n_in * n_out + n_out;
  }
  s[0] = a[0];
  s[1] = p.sizes[p.n_layers] > 1 ? a[1] : mk_t<T>(0.0);
}

// moments of the five stencil nodes (L, y), (L-1, y), (L-2, y), (L, y-1), (L, y+1)
// from their populations in[9n .. 9n+8]: mac[3n + {0, 1, 2}] = rho, u, v of node n
template <typename T>
__device__ __forceinline__ void stencil_macros(const T* in, T mac[15]) {
#pragma unroll
  for (int n = 0; n < 5; ++n) moments_g(in + 9 * n, mac[3 * n], mac[3 * n + 1], mac[3 * n + 2]);
}

// the six derivatives (p_x, u_x, v_x, p_y, u_y, v_y) of the east node from the
// stencil moments: one-sided second order in x, central in y, p = rho / 3
template <typename T>
__device__ __forceinline__ void features_g(const T mac[15], T fx[6]) {
  const double cs2 = 1.0 / 3.0;
  fx[0] = 0.5 * (3.0 * (cs2 * mac[0]) - 4.0 * (cs2 * mac[3]) + cs2 * mac[6]);
  fx[1] = 0.5 * (3.0 * mac[1] - 4.0 * mac[4] + mac[7]);
  fx[2] = 0.5 * (3.0 * mac[2] - 4.0 * mac[5] + mac[8]);
  fx[3] = 0.5 * (cs2 * mac[12] - cs2 * mac[9]);
  fx[4] = 0.5 * (mac[13] - mac[10]);
  fx[5] = 0.5 * (mac[14] - mac[11]);
}

// sigma and kappa2 of a node from its features: constants, or the tuner's
// sigma_max sigmoid(s_0) (and kappa2_max sigmoid(s_1) with two outputs)
template <typename T>
__device__ __forceinline__ void cbc_params_g(const SegParams& p, const T fx[6], T& sigma,
                                             T& kappa2) {
  sigma = mk_t<T>(p.sig_max);
  kappa2 = mk_t<T>(p.kap);
  if (p.n_layers > 0) {
    T s[2];
    tuner_g(p, fx, s);
    sigma = p.sig_max * sigmoid_g(s[0]);
    if (p.sizes[p.n_layers] > 1) kappa2 = p.kap * sigmoid_g(s[1]);
  }
}

// The east node (L, y) of one step from the stencil moments at t, the pulled
// known populations kn = f0(L, y), f1(L-1, y), f2(L, y-1), f4(L, y+1),
// f5(L-1, y-1), f8(L-1, y+1) and the node's sigma, kappa2: Eqs. 20-27, one
// Euler step, Zou & He with the prescribed state, the f_0 correction of Eq. 28
// (or the exact-mass one), then BGK.
template <typename T>
__device__ void east_core_g(const SegParams& p, const T mac[15], const T kn[6], T sigma,
                            T kappa2, T out[9]) {
  const double cs2 = 1.0 / 3.0;
  const double cs = sqrt(cs2);
  T fx[6];
  features_g(mac, fx);
  const T px = fx[0], ux = fx[1], vx = fx[2], py = fx[3], vy = fx[5];
  const T rho = mac[0], u0 = mac[1], v0 = mac[2];
  const T pL = cs2 * rho;
  const T L5 = (u0 + cs) * (px + rho * cs * ux);                 // Eq. 22
  const T L3 = u0 * vx;                                          // Eq. 21
  const T T1 = -(v0 * py + pL * vy - rho * cs * v0 * vy);        // Eq. 23
  const T T3 = -(v0 * vy + py / rho);                            // Eq. 24
  const T T5 = -(v0 * py + pL * vy + rho * cs * v0 * vy);        // Eq. 25
  const T kappa1 = sigma * p.kfac;                               // Eq. 27
  const T L1 = kappa1 * (pL - cs2 * p.rho_out) - kappa2 * T1 + T1;  // Eq. 26
  const T rn = rho + (-(L5 + L1) / (2.0 * cs2) + (T5 + T1) / (2.0 * cs2));       // Eq. 17
  const T un = u0 + (-(L5 - L1) / (2.0 * rho * cs) + (T5 - T1) / (2.0 * rho * cs));  // Eq. 18
  const T vn = v0 + (-L3 + T3);                                  // Eq. 19
  T g[9];
  g[0] = kn[0];
  g[1] = kn[1];
  g[2] = kn[2];
  g[4] = kn[3];
  g[5] = kn[4];
  g[8] = kn[5];
  T fe[9];
  feq_g(rn, un, vn, fe);
  const T half_t = 0.5 * ((g[4] - fe[4]) - (g[2] - fe[2]));
  g[3] = fe[3] + (g[1] - fe[1]);
  g[6] = fe[6] + (g[8] - fe[8]) + half_t;
  g[7] = fe[7] + (g[5] - fe[5]) - half_t;
  const T known = (g[0] + g[2] + g[4]) + 2.0 * (g[1] + g[5] + g[8]);
  if (p.exact) g[0] = g[0] + rn * (1.0 + un) - known;            // exact mass
  else g[0] = g[0] + rn - known / (1.0 + un);                    // Eq. 28
  bgk_g(g, p.omega, out);
}

// offset in a strip state of east input k of node y: k < 45 population k % 9 of
// stencil node k / 9, then the six known pulls
__device__ __forceinline__ int64_t east_input_offset(const SegParams& p, int y, int k) {
  const int W = p.W, ny = p.ny;
  const int64_t pl = node_plane(p);
  const int ym = wrap(y - 1, ny), yp = wrap(y + 1, ny);
  if (k < 45) {
    const int n = k / 9, i = k % 9;
    const int j = n == 1 ? W - 2 : (n == 2 ? W - 3 : W - 1);
    const int yy = n == 3 ? ym : (n == 4 ? yp : y);
    return i * pl + (int64_t)yy * W + j;
  }
  switch (k) {
    case 45: return 0 * pl + (int64_t)y * W + W - 1;
    case 46: return 1 * pl + (int64_t)y * W + W - 2;
    case 47: return 2 * pl + (int64_t)ym * W + W - 1;
    case 48: return 4 * pl + (int64_t)yp * W + W - 1;
    case 49: return 5 * pl + (int64_t)ym * W + W - 2;
    default: return 8 * pl + (int64_t)yp * W + W - 2;
  }
}

// index among the east node's inputs of the known pulled population i (-1: unknown)
__device__ __forceinline__ int known_input(int i) {
  switch (i) {
    case 0: return 45;
    case 1: return 46;
    case 2: return 47;
    case 4: return 48;
    case 5: return 49;
    case 8: return 50;
    default: return -1;
  }
}

// ---- kernels ----------------------------------------------------------------
__global__ void seg_init_kernel(const SegParams p) {
  const int s = blockIdx.y;
  const int64_t pl = node_plane(p);
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 9 * pl) return;
  const int j = (int)(k % p.W);
  const int64_t iy = k / p.W;            // i * ny + y
  const double* src = p.bank + (int64_t)p.init_idx[s] * 9 * p.ny * p.bank_w;
  hist_at(p, s, 0)[k] = src[iy * p.bank_w + (p.bank_w - p.W) + j];
}

// interior nodes (columns 0 .. W-2): pull and BGK
__global__ void seg_forward_kernel(const SegParams p, int t) {
  const int s = blockIdx.y;
  const int64_t pl = node_plane(p);
  const int wi = p.W - 1;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p.ny * wi) return;
  const int y = idx / wi, j = idx % wi;
  const double* A = hist_at(p, s, t);
  const double* A0 = hist_at(p, s, 0);
  double* B = hist_at(p, s, t + 1);
  double g[9], out[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int jsrc = j - cx(i);
    const int ysrc = wrap(y - cy(i), p.ny);
    g[i] = jsrc >= 0 ? A[i * pl + (int64_t)ysrc * p.W + jsrc]
                     : A0[i * pl + (int64_t)ysrc * p.W];     // frozen west edge
  }
  bgk_g<double>(g, p.omega, out);
  const int64_t o = (int64_t)y * p.W + j;
#pragma unroll
  for (int i = 0; i < 9; ++i) B[i * pl + o] = out[i];
}

// east nodes (column W-1): the characteristic outflow with the tuner
__global__ void seg_forward_east_kernel(const SegParams p, int t) {
  const int s = blockIdx.y;
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= p.ny) return;
  const int64_t pl = node_plane(p);
  const double* A = hist_at(p, s, t);
  double* B = hist_at(p, s, t + 1);
  double in[kEastInputs], mac[15], fx[6], sigma, kappa2, out[9];
  for (int k = 0; k < kEastInputs; ++k) in[k] = A[east_input_offset(p, y, k)];
  stencil_macros(in, mac);
  features_g(mac, fx);
  cbc_params_g(p, fx, sigma, kappa2);
  east_core_g<double>(p, mac, in + 45, sigma, kappa2, out);
  const int64_t o = (int64_t)y * p.W + p.W - 1;
#pragma unroll
  for (int i = 0; i < 9; ++i) B[i * pl + o] = out[i];
}

// loss of the batch (mean over segments) and lambda at t = n_t
__global__ void __launch_bounds__(128) seg_loss_kernel(const SegParams p) {
  __shared__ double red[128];
  const int s = blockIdx.y;
  const int64_t pl = node_plane(p);
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  double contrib = 0.0;
  if (idx < pl) {
    const int y = idx / p.W, j = idx % p.W;
    double lam[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (j >= p.W - p.n_t) {
      const double* A = hist_at(p, s, p.n_t);
      const double* R = p.bank + (int64_t)p.final_idx[s] * 9 * p.ny * p.bank_w;
      double f[9], fr[9];
      for (int i = 0; i < 9; ++i) {
        f[i] = A[i * pl + idx];
        fr[i] = R[((int64_t)i * p.ny + y) * p.bank_w + (p.bank_w - p.W) + j];
      }
      double rho, u, v, rr, ur, vr;
      moments_g(f, rho, u, v);
      moments_g(fr, rr, ur, vr);
      const double n = (double)p.n_t * p.ny;
      const double scale = 1.0 / p.n_seg;
      const double dr = rho - rr, du = u - ur, dv = v - vr;
      contrib = scale * (dr * dr / n + (du * du + dv * dv) / (2.0 * n));
      for (int i = 0; i < 9; ++i)
        lam[i] = scale * (2.0 * dr / n + (du * (cx(i) - u) + dv * (cy(i) - v)) / (n * rho));
    }
    for (int i = 0; i < 9; ++i) p.lam_in[(int64_t)s * 9 * pl + i * pl + idx] = lam[i];
  }
  red[threadIdx.x] = contrib;
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) p.loss_part[(int64_t)s * gridDim.x + blockIdx.x] = red[0];
}

// mu = J_BGK(p)^T lambda_{t+1} at every interior node (closed form)
__global__ void seg_adj_interior_kernel(const SegParams p, int t) {
  const int s = blockIdx.y;
  const int64_t pl = node_plane(p);
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= pl) return;
  const int y = idx / p.W, j = idx % p.W;
  if (j == p.W - 1) return;
  const double* A = hist_at(p, s, t);
  const double* A0 = hist_at(p, s, 0);
  const double* lam = p.lam_in + (int64_t)s * 9 * pl;
  double g[9], l[9];
  bool any = false;
  for (int i = 0; i < 9; ++i) {
    l[i] = lam[i * pl + idx];
    any |= l[i] != 0.0;
  }
  double* mu = p.mu + (int64_t)s * 9 * pl;
  if (!any) {
    for (int i = 0; i < 9; ++i) mu[i * pl + idx] = 0.0;
    return;
  }
  for (int i = 0; i < 9; ++i) {
    const int jsrc = j - cx(i);
    const int ysrc = wrap(y - cy(i), p.ny);
    g[i] = jsrc >= 0 ? A[i * pl + (int64_t)ysrc * p.W + jsrc] : A0[i * pl + (int64_t)ysrc * p.W];
  }
  double rho, u, v;
  moments_g(g, rho, u, v);
  // out_k = g_k - omega (g_k - w_k rho a_k), a_k = 1 + 3 cu + 4.5 cu^2 - 1.5 |u|^2
  double sr = 0.0, su = 0.0, sv = 0.0;
  const double usq = u * u + v * v;
  for (int k = 0; k < 9; ++k) {
    const double cu = cx(k) * u + cy(k) * v;
    const double wl = wgt<double>(k) * l[k];
    sr += wl * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
    su += wl * (3.0 * cx(k) + 9.0 * cu * cx(k) - 3.0 * u);
    sv += wl * (3.0 * cy(k) + 9.0 * cu * cy(k) - 3.0 * v);
  }
  // d rho / d g_i = 1, d u / d g_i = (c_ix - u) / rho; su, sv already carry rho / rho
  const double om = p.omega;
  for (int i = 0; i < 9; ++i)
    mu[i * pl + idx] = (1.0 - om) * l[i] + om * (sr + su * (cx(i) - u) + sv * (cy(i) - v));
}

// Input adjoints of lambda_{t+1}(L, y) . east_node, one warp per east node:
// lanes 0..5 differentiate the tuner along each feature (its Jacobian, once);
// lanes 0..22 differentiate the core along the 15 stencil moments, the 6 known
// pulls, sigma and kappa2 (forward mode); the moments' adjoints take the
// feature path (the features are linear in the moments) and become population
// adjoints through d(rho, u, v)/df.  Records (features, dL/dsigma, dL/dkappa2)
// feed the parameter gradient.
constexpr int kAdjWarps = 4;
constexpr int kAdjShared = 51 + 15 + 9 + 6 + 6 + 6 + 2 + 23 + 15;

__global__ void __launch_bounds__(32 * kAdjWarps) seg_adj_east_kernel(const SegParams p, int t) {
  __shared__ double sh[kAdjWarps][kAdjShared];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.y;
  const int y = blockIdx.x * kAdjWarps + warp;
  if (y >= p.ny) return;                     // whole warps only
  double* in = sh[warp];
  double* mac = in + 51;
  double* lam = mac + 15;
  double* fx = lam + 9;
  double* gs = fx + 6;
  double* gk = gs + 6;
  double* sk = gk + 6;
  double* a = sk + 2;
  double* mb = a + 23;
  const int64_t pl = node_plane(p);
  const double* A = hist_at(p, s, t);
  for (int k = lane; k < kEastInputs; k += 32) in[k] = A[east_input_offset(p, y, k)];
  if (lane < 9) lam[lane] = p.lam_in[(int64_t)s * 9 * pl + lane * pl + (int64_t)y * p.W + p.W - 1];
  __syncwarp();
  if (lane < 5) {
    double r, u, v;
    moments_g(in + 9 * lane, r, u, v);
    mac[3 * lane] = r;
    mac[3 * lane + 1] = u;
    mac[3 * lane + 2] = v;
  }
  __syncwarp();
  if (lane == 0) features_g(mac, fx);
  __syncwarp();
  if (lane < 6) {
    Dual xf[6];
    for (int k = 0; k < 6; ++k) xf[k] = {fx[k], k == lane ? 1.0 : 0.0};
    Dual sg, kp;
    cbc_params_g(p, xf, sg, kp);
    gs[lane] = sg.d;
    gk[lane] = kp.d;
    if (lane == 0) {
      sk[0] = sg.v;
      sk[1] = kp.v;
    }
  }
  __syncwarp();
  if (lane < 23) {
    Dual m[15], kn[6];
    for (int q = 0; q < 15; ++q) m[q] = {mac[q], q == lane ? 1.0 : 0.0};
    for (int q = 0; q < 6; ++q) kn[q] = {in[45 + q], 15 + q == lane ? 1.0 : 0.0};
    const Dual sg = {sk[0], lane == 21 ? 1.0 : 0.0};
    const Dual kp = {sk[1], lane == 22 ? 1.0 : 0.0};
    Dual out[9];
    east_core_g<Dual>(p, m, kn, sg, kp, out);
    double acc = 0.0;
    for (int i = 0; i < 9; ++i) acc += lam[i] * out[i].d;
    a[lane] = acc;
  }
  __syncwarp();
  if (lane < 15) {
    // feature path: fbar_f = dL/dsigma dsigma/dfx_f + dL/dkappa2 dkappa2/dfx_f,
    // times d fx_f / d mac_lane (the linear feature map, by one dual pass)
    Dual md[15], fd[6];
    for (int q = 0; q < 15; ++q) md[q] = {mac[q], q == lane ? 1.0 : 0.0};
    features_g(md, fd);
    double acc = a[lane];
    for (int f = 0; f < 6; ++f) acc += (a[21] * gs[f] + a[22] * gk[f]) * fd[f].d;
    mb[lane] = acc;
  }
  __syncwarp();
  double* e = p.east + ((int64_t)s * p.ny + y) * kEastInputs;
  for (int k = lane; k < kEastInputs; k += 32) {
    double v;
    if (k < 45) {
      const int n = k / 9, i = k % 9;
      const double rho = mac[3 * n], uu = mac[3 * n + 1], vv = mac[3 * n + 2];
      v = mb[3 * n] + (mb[3 * n + 1] * (cx(i) - uu) + mb[3 * n + 2] * (cy(i) - vv)) / rho;
    } else {
      v = a[15 + (k - 45)];
    }
    e[k] = v;
  }
  if (lane == 0) {
    double* rec = p.rec + (((int64_t)s * p.n_t + t) * p.ny + y) * kRecWidth;
    for (int k = 0; k < 6; ++k) rec[k] = fx[k];
    rec[6] = a[21];
    rec[7] = a[22];
  }
}

// lambda_t from the consumers' mu and the east nodes' input adjoints
__global__ void seg_gather_kernel(const SegParams p) {
  const int s = blockIdx.y;
  const int64_t pl = node_plane(p);
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= pl) return;
  const int y = idx / p.W, j = idx % p.W, W = p.W, ny = p.ny;
  const double* mu = p.mu + (int64_t)s * 9 * pl;
  const double* E = p.east + (int64_t)s * ny * kEastInputs;
  double* lam = p.lam_out + (int64_t)s * 9 * pl;
  const int yu = wrap(y + 1, ny), yd = wrap(y - 1, ny);
  for (int i = 0; i < 9; ++i) {
    double acc = 0.0;
    const int jc = j + cx(i), yc = wrap(y + cy(i), ny);
    if (jc >= 0 && jc <= W - 2) acc += mu[i * pl + (int64_t)yc * W + jc];
    else if (jc == W - 1) {
      const int k = known_input(i);
      if (k >= 0) acc += E[(int64_t)yc * kEastInputs + k];
    }
    if (j == W - 1)
      acc += E[(int64_t)y * kEastInputs + i] + E[(int64_t)yu * kEastInputs + 27 + i] +
             E[(int64_t)yd * kEastInputs + 36 + i];
    else if (j == W - 2)
      acc += E[(int64_t)y * kEastInputs + 9 + i];
    else if (j == W - 3)
      acc += E[(int64_t)y * kEastInputs + 18 + i];
    lam[i * pl + idx] = acc;
  }
}

// dL/dtheta: every record (features, dL/dsigma, dL/dkappa2) backpropagated
// through the tuner; per-block sums in record order, one partial per block
struct GradParams {
  int n_layers, sizes[LBM_MLP_MAX_LAYERS + 1], act, n_out;
  const double* net;
  const double* in_mean;
  const double* in_std;
  double sig_max, kap;
  int64_t n_params, n_rec;
  const double* rec;
  double* partial;       // [gridDim.x][n_params]
  int in_off[LBM_MLP_MAX_LAYERS], dl_off[LBM_MLP_MAX_LAYERS], per_rec;
};

__global__ void __launch_bounds__(kGradThreads) tuner_grad_kernel(const GradParams q) {
  extern __shared__ double sm[];
  double* gacc = sm;                                  // [n_params]
  double* buf = sm + ((q.n_params + 1) & ~int64_t(1)); // [kGradChunk][per_rec]
  for (int64_t k = threadIdx.x; k < q.n_params; k += blockDim.x) gacc[k] = 0.0;
  const int64_t chunks = (q.n_rec + kGradChunk - 1) / kGradChunk;
  for (int64_t c = blockIdx.x; c < chunks; c += gridDim.x) {
    const int64_t r0 = c * kGradChunk;
    const int64_t left = q.n_rec - r0;
    const int nr = left < kGradChunk ? (int)left : kGradChunk;
    __syncthreads();
    if ((int)threadIdx.x < nr) {
      const double* rc = q.rec + (r0 + threadIdx.x) * kRecWidth;
      double* mine = buf + threadIdx.x * q.per_rec;
      double a[kSegMaxW], z[LBM_MLP_MAX_LAYERS][kSegMaxW];
      for (int k = 0; k < 6; ++k) a[k] = (rc[k] - q.in_mean[k]) / q.in_std[k];
      int64_t off = 0;
      for (int l = 0; l < q.n_layers; ++l) {
        const int n_in = q.sizes[l], n_out = q.sizes[l + 1];
        const double* Wl = q.net + off;
        const double* bl = Wl + (int64_t)n_in * n_out;
        for (int k = 0; k < n_in; ++k) mine[q.in_off[l] + k] = a[k];
        double b[kSegMaxW];
        for (int j = 0; j < n_out; ++j) {
          double acc = bl[j];
          for (int k = 0; k < n_in; ++k) acc = acc + Wl[j * n_in + k] * a[k];
          z[l][j] = acc;
          b[j] = l == q.n_layers - 1 ? acc : act_g(acc, q.act);
        }
        for (int j = 0; j < n_out; ++j) a[j] = b[j];
        off += (int64_t)n_in * n_out + n_out;
      }
      // output deltas: sigma = sig_max sigmoid(s0), kappa2 = kap sigmoid(s1)
      double dl[kSegMaxW];
      {
        const double s0 = 1.0 / (1.0 + exp(-a[0]));
        dl[0] = rc[6] * q.sig_max * s0 * (1.0 - s0);
        if (q.n_out > 1) {
          const double s1 = 1.0 / (1.0 + exp(-a[1]));
          dl[1] = rc[7] * q.kap * s1 * (1.0 - s1);
        }
      }
      int64_t offs[LBM_MLP_MAX_LAYERS];
      {
        int64_t o2 = 0;
        for (int l = 0; l < q.n_layers; ++l) {
          offs[l] = o2;
          o2 += (int64_t)q.sizes[l] * q.sizes[l + 1] + q.sizes[l + 1];
        }
      }
      for (int l = q.n_layers - 1; l >= 0; --l) {
        const int n_in = q.sizes[l], n_out = q.sizes[l + 1];
        for (int j = 0; j < n_out; ++j) mine[q.dl_off[l] + j] = dl[j];
        if (l == 0) break;
        const double* Wl = q.net + offs[l];
        double nd[kSegMaxW];
        for (int k = 0; k < n_in; ++k) {
          double acc = 0.0;
          for (int j = 0; j < n_out; ++j) acc += Wl[j * n_in + k] * dl[j];
          const double zz = z[l - 1][k];
          double dz;
          if (q.act == 0) {
            const double th = tanh(zz);
            dz = 1.0 - th * th;
          } else {
            dz = zz > 0.0 ? 1.0 : 0.01;
          }
          nd[k] = acc * dz;
        }
        for (int k = 0; k < n_in; ++k) dl[k] = nd[k];
      }
    }
    __syncthreads();
    // parameter sums over this chunk's records, in record order
    int64_t off = 0;
    for (int l = 0; l < q.n_layers; ++l) {
      const int n_in = q.sizes[l], n_out = q.sizes[l + 1];
      const int64_t nw = (int64_t)n_in * n_out;
      for (int64_t k = threadIdx.x; k < nw + n_out; k += blockDim.x) {
        double acc = 0.0;
        if (k < nw) {
          const int j = (int)(k / n_in), kk = (int)(k % n_in);
          for (int r = 0; r < nr; ++r) {
            const double* m = buf + r * q.per_rec;
            acc += m[q.dl_off[l] + j] * m[q.in_off[l] + kk];
          }
        } else {
          const int j = (int)(k - nw);
          for (int r = 0; r < nr; ++r) acc += buf[r * q.per_rec + q.dl_off[l] + j];
        }
        gacc[off + k] += acc;
      }
      off += nw + n_out;
    }
  }
  __syncthreads();
  for (int64_t k = threadIdx.x; k < q.n_params; k += blockDim.x)
    q.partial[(int64_t)blockIdx.x * q.n_params + k] = gacc[k];
}

// grad[k] = sum over blocks in order; loss = sum of the loss partials in order
__global__ void sum_partials_kernel(const double* part, int nb, int64_t n, double* out) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double acc = 0.0;
  for (int b = 0; b < nb; ++b) acc += part[(int64_t)b * n + k];
  out[k] = acc;
}

__global__ void sum_loss_kernel(const double* part, int64_t n, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double acc = 0.0;
  for (int64_t k = 0; k < n; ++k) acc += part[k];
  *out = acc;
}

// Adam (Kingma & Ba 2015); c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t)
__global__ void adam_kernel(double* prm, double* m, double* v, const double* g, int64_t n,
                            double lr, double b1, double b2, double eps, double c1, double c2) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  m[k] = b1 * m[k] + (1.0 - b1) * g[k];
  v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k];
  const double mh = m[k] * c1, vh = v[k] * c2;
  prm[k] = prm[k] - lr * mh / (sqrt(vh) + eps);
}

// Mean and population standard deviation of the six tuner features over the
// east nodes of every bank state (one block, fixed summation order).
__global__ void __launch_bounds__(256) feature_stats_kernel(const double* bank, int n_states,
                                                            int ny, int bank_w, double* out) {
  __shared__ double red[6][256];
  __shared__ double mean[6];
  const int64_t n = (int64_t)n_states * ny;
  for (int pass = 0; pass < 2; ++pass) {
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
      const int st = (int)(k / ny), y = (int)(k % ny);
      const double* A = bank + (int64_t)st * 9 * ny * bank_w;
      const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
      const int js[5] = {bank_w - 1, bank_w - 2, bank_w - 3, bank_w - 1, bank_w - 1};
      const int ys[5] = {y, y, y, ym, yp};
      double in[45], mac[15], fx[6];
      for (int q = 0; q < 5; ++q)
        for (int i = 0; i < 9; ++i) in[9 * q + i] = A[((int64_t)i * ny + ys[q]) * bank_w + js[q]];
      stencil_macros(in, mac);
      features_g(mac, fx);
      for (int f = 0; f < 6; ++f) {
        const double d = pass == 0 ? fx[f] : fx[f] - mean[f];
        acc[f] += pass == 0 ? d : d * d;
      }
    }
    for (int f = 0; f < 6; ++f) red[f][threadIdx.x] = acc[f];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w)
        for (int f = 0; f < 6; ++f) red[f][threadIdx.x] += red[f][threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x < 6) {
      const double m = red[threadIdx.x][0] / (double)n;
      if (pass == 0) mean[threadIdx.x] = m;
      else out[6 + threadIdx.x] = sqrt(m);
      if (pass == 0) out[threadIdx.x] = m;
    }
    __syncthreads();
  }
}

template <typename S>
__global__ void copy_columns_kernel(const S* src, int ny, int64_t pitch, int64_t plane, int x0,
                                    int width, double* out) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)9 * ny * width;
  if (k >= n) return;
  const int j = (int)(k % width);
  const int64_t iy = k / width;
  const int y = (int)(iy % ny), i = (int)(iy / ny);
  out[k] = (double)to_r<double>(src[i * plane + (int64_t)y * pitch + x0 + j]) + wgt<double>(i);
}

struct Scratch {
  std::vector<void*> ptrs;
  ~Scratch() {
    for (void* q : ptrs) cudaFree(q);
  }
  template <typename T>
  T* get(size_t n) {
    void* q = nullptr;
    ck(cudaMalloc(&q, std::max<size_t>(n * sizeof(T), 16)), "cudaMalloc");
    ptrs.push_back(q);
    return static_cast<T*>(q);
  }
};

lbm_status seg_fail(lbm_status st, const char* msg) {
  set_last_error(msg);
  return st;
}

int64_t tuner_params(const lbm_mlp* t) {
  int64_t np = 0;
  for (int l = 0; l < t->n_layers; ++l) np += (int64_t)t->sizes[l] * t->sizes[l + 1] + t->sizes[l + 1];
  return np;
}

lbm_status check_segments(const lbm_cbc_segments* g, const lbm_mlp* tuner, int64_t* np_out) {
  if (!g || !tuner) return seg_fail(LBM_ERR_ARG, "segments and tuner must be non-NULL");
  if (g->n_t < 1) return seg_fail(LBM_ERR_ARG, "n_t must be >= 1");
  const int W = std::max(2 * g->n_t, 3);
  if (g->ny < 3 || g->ny > 65535) return seg_fail(LBM_ERR_ARG, "ny must be in [3, 65535]");
  if (g->nx < W + 1) return seg_fail(LBM_ERR_ARG, "nx must be >= max(2 n_t, 3) + 1");
  if (g->bank_width < W || g->bank_width > g->nx)
    return seg_fail(LBM_ERR_ARG, "bank_width must be in [max(2 n_t, 3), nx]");
  if (!g->bank || g->n_states < 1) return seg_fail(LBM_ERR_ARG, "bank must hold >= 1 state");
  if (!(g->tau > 0.5) || !std::isfinite(g->tau)) return seg_fail(LBM_ERR_ARG, "tau must be > 1/2");
  if (!std::isfinite(g->sigma) || !std::isfinite(g->kappa2) || !std::isfinite(g->mach) ||
      !std::isfinite(g->rho_out) || g->length < 0.0 || !std::isfinite(g->length))
    return seg_fail(LBM_ERR_ARG, "non-finite CBC setting");
  if (tuner->n_layers < 1 || tuner->n_layers > 3)
    return seg_fail(LBM_ERR_ARG, "the tuner has 1..3 layers");
  if (tuner->sizes[0] != 6) return seg_fail(LBM_ERR_ARG, "the tuner has 6 inputs");
  const int n_out = tuner->sizes[tuner->n_layers];
  if (n_out != 1 && n_out != 2) return seg_fail(LBM_ERR_ARG, "the tuner has 1 or 2 outputs");
  for (int l = 1; l < tuner->n_layers; ++l)
    if (tuner->sizes[l] < 1 || tuner->sizes[l] > kSegMaxW)
      return seg_fail(LBM_ERR_ARG, "tuner hidden layers have 1..32 units");
  if (tuner->act != 0 && tuner->act != 1) return seg_fail(LBM_ERR_ARG, "act must be 0 or 1");
  for (int k = 0; k < 6; ++k) {
    if (tuner->in_std && !(tuner->in_std[k] > 0.f)) return seg_fail(LBM_ERR_ARG, "in_std must be > 0");
    if (tuner->in_mean && !std::isfinite(tuner->in_mean[k]))
      return seg_fail(LBM_ERR_ARG, "in_mean must be finite");
  }
  *np_out = tuner_params(tuner);
  return LBM_OK;
}

// One loss + gradient evaluation of a batch of segments (device indices) at the
// parameters d_net; grad (device, n_params) and loss (device, 1) are written.
class SegmentRunner {
 public:
  SegmentRunner(const lbm_cbc_segments* g, const lbm_mlp* tuner, int64_t np, int max_batch,
                cudaStream_t st)
      : st_(st) {
    p_ = SegParams{};
    p_.ny = g->ny;
    p_.n_t = g->n_t;
    p_.W = std::max(2 * g->n_t, 3);
    p_.bank_w = g->bank_width;
    p_.omega = 1.0 / g->tau;
    p_.rho_out = g->rho_out;
    p_.sig_max = g->sigma;
    p_.kap = g->kappa2;
    const double cs = std::sqrt(1.0 / 3.0);
    const double length = g->length > 0.0 ? g->length : (double)g->nx;
    p_.kfac = (1.0 - g->mach * g->mach) * cs / length;
    p_.exact = g->exact_mass ? 1 : 0;
    p_.n_layers = tuner->n_layers;
    for (int l = 0; l <= LBM_MLP_MAX_LAYERS; ++l)
      p_.sizes[l] = l <= tuner->n_layers ? tuner->sizes[l] : 0;
    p_.act = tuner->act;
    p_.n_params = np;
    p_.bank = g->bank;
    const int64_t pl = (int64_t)p_.ny * p_.W;
    d_net_ = sc_.get<double>(np);
    d_norm_ = sc_.get<double>(12);
    std::vector<double> norm(12);
    for (int k = 0; k < 6; ++k) {
      norm[k] = tuner->in_mean ? tuner->in_mean[k] : 0.0;
      norm[6 + k] = tuner->in_std ? tuner->in_std[k] : 1.0;
    }
    ck(cudaMemcpyAsync(d_norm_, norm.data(), 12 * 8, cudaMemcpyHostToDevice, st_), "copy");
    p_.net = d_net_;
    p_.in_mean = d_norm_;
    p_.in_std = d_norm_ + 6;
    p_.init_idx = d_init_ = sc_.get<int>(max_batch);
    p_.final_idx = d_final_ = sc_.get<int>(max_batch);
    p_.hist = sc_.get<double>((size_t)max_batch * (p_.n_t + 1) * 9 * pl);
    p_.lam_in = sc_.get<double>((size_t)max_batch * 9 * pl);
    p_.lam_out = sc_.get<double>((size_t)max_batch * 9 * pl);
    p_.mu = sc_.get<double>((size_t)max_batch * 9 * pl);
    p_.east = sc_.get<double>((size_t)max_batch * p_.ny * kEastInputs);
    p_.rec = sc_.get<double>((size_t)max_batch * p_.n_t * p_.ny * kRecWidth);
    loss_blocks_ = (int)((pl + 127) / 128);
    p_.loss_part = sc_.get<double>((size_t)max_batch * loss_blocks_);
    grad_part_ = sc_.get<double>((size_t)kGradBlocks * np);
    // gradient kernel layout: per record the inputs of every layer, then the deltas
    gq_ = GradParams{};
    gq_.n_layers = p_.n_layers;
    for (int l = 0; l <= LBM_MLP_MAX_LAYERS; ++l) gq_.sizes[l] = p_.sizes[l];
    gq_.act = p_.act;
    gq_.n_out = p_.sizes[p_.n_layers];
    gq_.sig_max = p_.sig_max;
    gq_.kap = p_.kap;
    gq_.n_params = np;
    int o = 0;
    for (int l = 0; l < p_.n_layers; ++l) {
      gq_.in_off[l] = o;
      o += p_.sizes[l];
    }
    for (int l = 0; l < p_.n_layers; ++l) {
      gq_.dl_off[l] = o;
      o += p_.sizes[l + 1];
    }
    gq_.per_rec = o;
    grad_smem_ = (size_t)(((np + 1) & ~int64_t(1)) + (int64_t)kGradChunk * o) * sizeof(double);
    ck(cudaFuncSetAttribute(tuner_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)grad_smem_), "smem attribute");
  }

  double* net() { return d_net_; }

  // indices: device int arrays already filled for n segments
  void run(int n, double* d_grad, double* d_loss) {
    SegParams p = p_;
    p.n_seg = n;
    const int64_t pl = (int64_t)p.ny * p.W;
    const dim3 gn((unsigned)((pl + 127) / 128), (unsigned)n);
    const dim3 gi((unsigned)((9 * pl + 127) / 128), (unsigned)n);
    seg_init_kernel<<<gi, 128, 0, st_>>>(p);
    const dim3 gf((unsigned)((p.ny * (p.W - 1) + 127) / 128), (unsigned)n);
    const dim3 ge((unsigned)((p.ny + 63) / 64), (unsigned)n);
    for (int t = 0; t < p.n_t; ++t) {
      seg_forward_kernel<<<gf, 128, 0, st_>>>(p, t);
      seg_forward_east_kernel<<<ge, 64, 0, st_>>>(p, t);
    }
    seg_loss_kernel<<<gn, 128, 0, st_>>>(p);
    sum_loss_kernel<<<1, 32, 0, st_>>>(p.loss_part, (int64_t)n * loss_blocks_, d_loss);
    for (int t = p.n_t - 1; t >= 0; --t) {
      seg_adj_interior_kernel<<<gn, 128, 0, st_>>>(p, t);
      seg_adj_east_kernel<<<dim3((unsigned)((p.ny + kAdjWarps - 1) / kAdjWarps), (unsigned)n),
                            32 * kAdjWarps, 0, st_>>>(p, t);
      if (t > 0) {
        seg_gather_kernel<<<gn, 128, 0, st_>>>(p);
        std::swap(p.lam_in, p.lam_out);
      }
    }
    GradParams q = gq_;
    q.net = d_net_;
    q.in_mean = d_norm_;
    q.in_std = d_norm_ + 6;
    q.n_rec = (int64_t)n * p.n_t * p.ny;
    q.rec = p.rec;
    q.partial = grad_part_;
    tuner_grad_kernel<<<kGradBlocks, kGradThreads, grad_smem_, st_>>>(q);
    sum_partials_kernel<<<(unsigned)((q.n_params + 127) / 128), 128, 0, st_>>>(
        grad_part_, kGradBlocks, q.n_params, d_grad);
    ck(cudaGetLastError(), "segment launches");
  }

  int* init_idx() { return d_init_; }
  int* final_idx() { return d_final_; }

 private:
  cudaStream_t st_;
  Scratch sc_;
  SegParams p_;
  GradParams gq_;
  double* d_net_ = nullptr;
  double* d_norm_ = nullptr;
  int* d_init_ = nullptr;
  int* d_final_ = nullptr;
  double* grad_part_ = nullptr;
  int loss_blocks_ = 0;
  size_t grad_smem_ = 0;
};

lbm_status check_indices(const lbm_cbc_segments* g) {
  if (g->n_seg < 1 || g->n_seg > 65535 || !g->init_state || !g->final_state)
    return seg_fail(LBM_ERR_ARG, "n_seg in [1, 65535] and the index arrays are required");
  for (int k = 0; k < g->n_seg; ++k)
    if (g->init_state[k] < 0 || g->init_state[k] >= g->n_states || g->final_state[k] < 0 ||
        g->final_state[k] >= g->n_states)
      return seg_fail(LBM_ERR_ARG, "state index out of range");
  return LBM_OK;
}

}  // namespace
}  // namespace lbm

extern "C" {

lbm_status lbm_copy_columns(lbm_sim* s, int32_t x0, int32_t width, double* dev_out) {
  using namespace lbm;
  if (!s || !s->buf[0]) return seg_fail(LBM_ERR_STATE, "sim is not initialised");
  if (!dev_out) return seg_fail(LBM_ERR_ARG, "dev_out is NULL");
  if (width < 1 || x0 < 0 || (int64_t)x0 + width > s->nx)
    return seg_fail(LBM_ERR_ARG, "columns out of range");
  try {
    const int64_t n = (int64_t)9 * s->ny * width;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (s->prec == LBM_FP64)
      copy_columns_kernel<double><<<blocks, 256, 0, s->stream>>>(
          (const double*)s->buf[s->cur], s->ny, s->pitch, s->plane, x0, width, dev_out);
    else if (s->prec == LBM_FP32)
      copy_columns_kernel<float><<<blocks, 256, 0, s->stream>>>(
          (const float*)s->buf[s->cur], s->ny, s->pitch, s->plane, x0, width, dev_out);
    else
      copy_columns_kernel<__half><<<blocks, 256, 0, s->stream>>>(
          (const __half*)s->buf[s->cur], s->ny, s->pitch, s->plane, x0, width, dev_out);
    ck(cudaGetLastError(), "column copy");
  } catch (const CudaError& ce) {
    set_last_error(std::string(ce.what) + ": " + cudaGetErrorString(ce.e));
    return LBM_ERR_CUDA;
  }
  return LBM_OK;
}

lbm_status lbm_cbc_feature_stats(const lbm_cbc_segments* g, float* in_mean, float* in_std) {
  using namespace lbm;
  if (!g || !in_mean || !in_std) return seg_fail(LBM_ERR_ARG, "segs, in_mean and in_std are required");
  if (!g->bank || g->n_states < 1) return seg_fail(LBM_ERR_ARG, "bank must hold >= 1 state");
  if (g->ny < 3 || g->bank_width < 3) return seg_fail(LBM_ERR_ARG, "ny and bank_width must be >= 3");
  try {
    cudaStream_t st = static_cast<cudaStream_t>(g->stream);
    Scratch sc;
    double* d_out = sc.get<double>(12);
    feature_stats_kernel<<<1, 256, 0, st>>>(g->bank, g->n_states, g->ny, g->bank_width, d_out);
    ck(cudaGetLastError(), "feature statistics");
    double h[12];
    ck(cudaMemcpyAsync(h, d_out, sizeof h, cudaMemcpyDeviceToHost, st), "copy");
    ck(cudaStreamSynchronize(st), "sync");
    for (int k = 0; k < 6; ++k) {
      in_mean[k] = (float)h[k];
      in_std[k] = h[6 + k] < 1e-12 || !std::isfinite(h[6 + k]) ? 1.f : (float)h[6 + k];
    }
  } catch (const CudaError& ce) {
    set_last_error(std::string(ce.what) + ": " + cudaGetErrorString(ce.e));
    return LBM_ERR_CUDA;
  }
  return LBM_OK;
}

lbm_status lbm_cbc_segment_grad(const lbm_cbc_segments* g, const lbm_mlp* tuner,
                                const double* params, double* loss, double* grad) {
  using namespace lbm;
  int64_t np = 0;
  if (lbm_status st = check_segments(g, tuner, &np)) return st;
  if (lbm_status st = check_indices(g)) return st;
  if (!params || !loss) return seg_fail(LBM_ERR_ARG, "params and loss must be non-NULL");
  for (int64_t k = 0; k < np; ++k)
    if (!std::isfinite(params[k])) return seg_fail(LBM_ERR_ARG, "non-finite parameter");
  try {
    cudaStream_t st = static_cast<cudaStream_t>(g->stream);
    SegmentRunner run(g, tuner, np, g->n_seg, st);
    Scratch sc;
    double* d_grad = sc.get<double>(np);
    double* d_loss = sc.get<double>(1);
    ck(cudaMemcpyAsync(run.net(), params, np * 8, cudaMemcpyHostToDevice, st), "copy");
    ck(cudaMemcpyAsync(run.init_idx(), g->init_state, g->n_seg * 4, cudaMemcpyHostToDevice, st),
       "copy");
    ck(cudaMemcpyAsync(run.final_idx(), g->final_state, g->n_seg * 4, cudaMemcpyHostToDevice, st),
       "copy");
    run.run(g->n_seg, d_grad, d_loss);
    ck(cudaMemcpyAsync(loss, d_loss, 8, cudaMemcpyDeviceToHost, st), "copy");
    if (grad) ck(cudaMemcpyAsync(grad, d_grad, np * 8, cudaMemcpyDeviceToHost, st), "copy");
    ck(cudaStreamSynchronize(st), "sync");
  } catch (const CudaError& ce) {
    set_last_error(std::string(ce.what) + ": " + cudaGetErrorString(ce.e));
    return ce.e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
  }
  return LBM_OK;
}

lbm_status lbm_cbc_tuner_train(const lbm_cbc_segments* g, const lbm_mlp* tuner,
                               const int32_t* order, int32_t batch, int64_t n_steps,
                               const lbm_train_opts* o, double* params, double* adam_m,
                               double* adam_v, double* loss_log) {
  using namespace lbm;
  int64_t np = 0;
  if (lbm_status st = check_segments(g, tuner, &np)) return st;
  if (lbm_status st = check_indices(g)) return st;
  if (!order || !o || !params) return seg_fail(LBM_ERR_ARG, "order, opts and params are required");
  if (batch < 1 || batch > 65535 || n_steps < 0)
    return seg_fail(LBM_ERR_ARG, "batch in [1, 65535] and n_steps >= 0");
  for (int64_t k = 0; k < (int64_t)batch * n_steps; ++k)
    if (order[k] < 0 || order[k] >= g->n_seg) return seg_fail(LBM_ERR_ARG, "segment index out of range");
  if (!(o->lr > 0) || !(o->eps > 0) || !(o->beta1 >= 0 && o->beta1 < 1) ||
      !(o->beta2 >= 0 && o->beta2 < 1) || o->adam_t0 < 0)
    return seg_fail(LBM_ERR_ARG, "Adam needs lr > 0, eps > 0, 0 <= beta1, beta2 < 1, adam_t0 >= 0");
  for (int64_t k = 0; k < np; ++k)
    if (!std::isfinite(params[k])) return seg_fail(LBM_ERR_ARG, "non-finite parameter");
  if (n_steps == 0) return LBM_OK;
  try {
    cudaStream_t st = static_cast<cudaStream_t>(o->stream ? o->stream : g->stream);
    SegmentRunner run(g, tuner, np, batch, st);
    Scratch sc;
    double* d_grad = sc.get<double>(np);
    double* d_m = sc.get<double>(np);
    double* d_v = sc.get<double>(np);
    double* d_loss = sc.get<double>(n_steps);
    ck(cudaMemcpyAsync(run.net(), params, np * 8, cudaMemcpyHostToDevice, st), "copy");
    if (adam_m) ck(cudaMemcpyAsync(d_m, adam_m, np * 8, cudaMemcpyHostToDevice, st), "copy");
    else ck(cudaMemsetAsync(d_m, 0, np * 8, st), "memset");
    if (adam_v) ck(cudaMemcpyAsync(d_v, adam_v, np * 8, cudaMemcpyHostToDevice, st), "copy");
    else ck(cudaMemsetAsync(d_v, 0, np * 8, st), "memset");
    // batch b's bank indices, gathered on the host (tiny)
    std::vector<int> bi((size_t)batch * n_steps), bf((size_t)batch * n_steps);
    for (int64_t k = 0; k < (int64_t)batch * n_steps; ++k) {
      bi[k] = g->init_state[order[k]];
      bf[k] = g->final_state[order[k]];
    }
    int* d_bi = sc.get<int>(bi.size());
    int* d_bf = sc.get<int>(bf.size());
    ck(cudaMemcpyAsync(d_bi, bi.data(), bi.size() * 4, cudaMemcpyHostToDevice, st), "copy");
    ck(cudaMemcpyAsync(d_bf, bf.data(), bf.size() * 4, cudaMemcpyHostToDevice, st), "copy");
    for (int64_t k = 0; k < n_steps; ++k) {
      ck(cudaMemcpyAsync(run.init_idx(), d_bi + k * batch, batch * 4, cudaMemcpyDeviceToDevice, st),
         "copy");
      ck(cudaMemcpyAsync(run.final_idx(), d_bf + k * batch, batch * 4, cudaMemcpyDeviceToDevice,
                         st), "copy");
      run.run(batch, d_grad, d_loss + k);
      const double tt = (double)(o->adam_t0 + k + 1);
      const double c1 = 1.0 / (1.0 - std::pow(o->beta1, tt));
      const double c2 = 1.0 / (1.0 - std::pow(o->beta2, tt));
      adam_kernel<<<(unsigned)((np + 127) / 128), 128, 0, st>>>(run.net(), d_m, d_v, d_grad, np,
                                                                o->lr, o->beta1, o->beta2, o->eps,
                                                                c1, c2);
      ck(cudaGetLastError(), "adam launch");
    }
    ck(cudaMemcpyAsync(params, run.net(), np * 8, cudaMemcpyDeviceToHost, st), "copy");
    if (adam_m) ck(cudaMemcpyAsync(adam_m, d_m, np * 8, cudaMemcpyDeviceToHost, st), "copy");
    if (adam_v) ck(cudaMemcpyAsync(adam_v, d_v, np * 8, cudaMemcpyDeviceToHost, st), "copy");
    if (loss_log) ck(cudaMemcpyAsync(loss_log, d_loss, n_steps * 8, cudaMemcpyDeviceToHost, st), "copy");
    ck(cudaStreamSynchronize(st), "sync");
  } catch (const CudaError& ce) {
    set_last_error(std::string(ce.what) + ": " + cudaGetErrorString(ce.e));
    return ce.e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
  }
  return LBM_OK;
}

}  // extern "C"
