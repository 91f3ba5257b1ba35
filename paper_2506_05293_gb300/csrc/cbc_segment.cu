// Training of the CBC tuner through short simulation segments (Sec. 4.2 and
// its tuning-procedure figure): forward segments on east strips, their loss,
// the reverse (adjoint) pass and Adam, on the device.
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
// States, adjoints and the tuner run in the compute type R: double, or float
// on shifted populations h = f - w with densities carried as rho - 1 (the
// deviations FP32 keeps to full relative precision; GB300 issues FP32 far
// faster than FP64).  The loss, the parameter sums and Adam are FP64.
//
// Reverse pass, step t+1 -> t, given lambda_{t+1} = dL/dh(t+1):
//  * interior node: h(t+1) = BGK(p), p_i = h_i(x - c_i, t); mu = J_BGK(p)^T lambda
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
// record through the tuner, sums them per chunk of records and per block and
// then over blocks in a fixed order.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <memory>
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
constexpr int kAdjWarps = 4;              // east nodes per block of the east adjoint
constexpr int kAdjShared = 51 + 15 + 9 + 6 + 6 + 6 + 2 + 23 + 15;

// ---- forward-mode dual numbers and scalar helpers ----------------------------
template <typename R>
struct DualT {
  R v, d;
};
template <typename T> struct ScalarOf { using type = T; };
template <typename R> struct ScalarOf<DualT<R>> { using type = R; };

template <typename R>
__device__ __forceinline__ DualT<R> operator+(DualT<R> a, DualT<R> b) { return {a.v + b.v, a.d + b.d}; }
template <typename R>
__device__ __forceinline__ DualT<R> operator-(DualT<R> a, DualT<R> b) { return {a.v - b.v, a.d - b.d}; }
template <typename R>
__device__ __forceinline__ DualT<R> operator-(DualT<R> a) { return {-a.v, -a.d}; }
template <typename R>
__device__ __forceinline__ DualT<R> operator*(DualT<R> a, DualT<R> b) {
  return {a.v * b.v, a.d * b.v + a.v * b.d};
}
template <typename R>
__device__ __forceinline__ DualT<R> operator/(DualT<R> a, DualT<R> b) {
  const R q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
template <typename R>
__device__ __forceinline__ DualT<R> operator+(DualT<R> a, R b) { return {a.v + b, a.d}; }
template <typename R>
__device__ __forceinline__ DualT<R> operator+(R a, DualT<R> b) { return {a + b.v, b.d}; }
template <typename R>
__device__ __forceinline__ DualT<R> operator-(DualT<R> a, R b) { return {a.v - b, a.d}; }
template <typename R>
__device__ __forceinline__ DualT<R> operator*(DualT<R> a, R b) { return {a.v * b, a.d * b}; }
template <typename R>
__device__ __forceinline__ DualT<R> operator*(R a, DualT<R> b) { return {a * b.v, a * b.d}; }
template <typename R>
__device__ __forceinline__ DualT<R> operator/(DualT<R> a, R b) { return {a.v / b, a.d / b}; }

template <typename T>
__device__ __forceinline__ T mk_t(typename ScalarOf<T>::type v) { return T{v}; }
template <>
__device__ __forceinline__ DualT<float> mk_t<DualT<float>>(float v) { return {v, 0.f}; }
template <>
__device__ __forceinline__ DualT<double> mk_t<DualT<double>>(double v) { return {v, 0.0}; }

__device__ __forceinline__ float value(float a) { return a; }
__device__ __forceinline__ double value(double a) { return a; }
template <typename R>
__device__ __forceinline__ R value(DualT<R> a) { return a.v; }

__device__ __forceinline__ float tanh_s(float a) { return tanhf(a); }
__device__ __forceinline__ double tanh_s(double a) { return tanh(a); }
__device__ __forceinline__ float exp_s(float a) { return expf(a); }
__device__ __forceinline__ double exp_s(double a) { return exp(a); }

template <typename R>
__device__ __forceinline__ R tanh_g(R a) { return tanh_s(a); }
template <typename R>
__device__ __forceinline__ DualT<R> tanh_g(DualT<R> a) {
  const R t = tanh_s(a.v);
  return {t, (R(1) - t * t) * a.d};
}
template <typename R>
__device__ __forceinline__ R sigmoid_g(R a) { return R(1) / (R(1) + exp_s(-a)); }
template <typename R>
__device__ __forceinline__ DualT<R> sigmoid_g(DualT<R> a) {
  const R s = R(1) / (R(1) + exp_s(-a.v));
  return {s, s * (R(1) - s) * a.d};
}
template <typename T>
__device__ __forceinline__ T act_g(T a, int act) {
  using S = typename ScalarOf<T>::type;
  if (act == 0) return tanh_g(a);
  return value(a) > S(0) ? a : a * S(0.01);   // LeakyReLU, slope 0.01
}

template <typename R>
struct SegParams {
  int n_seg, ny, W, n_t, bank_w;
  R omega, drho_out, sig_max, kap, kfac;     // drho_out = rho_out - 1
  int exact;
  // tuner: per layer W (n_out x n_in, row-major) then b; z-scored inputs
  int n_layers, sizes[LBM_MLP_MAX_LAYERS + 1], act;
  const R* net;
  const R* in_mean;
  const R* in_std;
  // data
  const double* bank;     // [n_states][9][ny][bank_w] populations f
  const int* init_idx;    // [n_seg]
  const int* final_idx;   // [n_seg]
  R* hist;                // [n_seg][n_t + 1][9][ny][W]   h = f - w
  R* lam_in;              // [n_seg][9][ny][W]   lambda_{t+1}
  R* lam_out;             // [n_seg][9][ny][W]   lambda_t
  R* mu;                  // [n_seg][9][ny][W]
  R* east;                // [n_seg][ny][kEastInputs]
  R* rec;                 // [n_seg][n_t][ny][kRecWidth]
  double* loss_part;      // per block of the loss kernel
};

template <typename R>
__device__ __forceinline__ int64_t node_plane(const SegParams<R>& p) { return (int64_t)p.ny * p.W; }
template <typename R>
__device__ __forceinline__ R* hist_at(const SegParams<R>& p, int s, int t) {
  return p.hist + ((int64_t)s * (p.n_t + 1) + t) * 9 * node_plane(p);
}
__device__ __forceinline__ int wrap(int y, int ny) { return y < 0 ? y + ny : (y >= ny ? y - ny : y); }

// rho - 1, u, v of shifted populations (Eq. 4)
template <typename T>
__device__ __forceinline__ void moments_h(const T h[9], T& dr, T& u, T& v) {
  using S = typename ScalarOf<T>::type;
  dr = h[0] + h[1] + h[2] + h[3] + h[4] + h[5] + h[6] + h[7] + h[8];
  const T jx = h[1] - h[3] + h[5] - h[6] - h[7] + h[8];
  const T jy = h[2] - h[4] + h[5] + h[6] - h[7] - h[8];
  const T rho = S(1) + dr;
  u = jx / rho;
  v = jy / rho;
}

// Eq. 3 shifted: f_i^eq - w_i = w_i (rho - 1 + rho (3 cu + 4.5 cu^2 - 1.5 |u|^2))
template <typename T>
__device__ __forceinline__ void heq_g(T dr, T u, T v, T out[9]) {
  using S = typename ScalarOf<T>::type;
  const T usq = u * u + v * v;
  const T rho = S(1) + dr;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const T cu = S(cx(i)) * u + S(cy(i)) * v;
    out[i] = wgt<S>(i) * (dr + rho * (S(3) * cu + S(4.5) * (cu * cu) - S(1.5) * usq));
  }
}

// Eq. 2 on shifted populations
template <typename T>
__device__ __forceinline__ void bgk_h(const T h[9], typename ScalarOf<T>::type omega, T out[9]) {
  T dr, u, v, fe[9];
  moments_h(h, dr, u, v);
  heq_g(dr, u, v, fe);
#pragma unroll
  for (int i = 0; i < 9; ++i) out[i] = h[i] - omega * (h[i] - fe[i]);
}

template <typename T, typename R>
__device__ void tuner_g(const SegParams<R>& p, const T x[6], T s[2]) {
  T a[kSegMaxW], b[kSegMaxW];
  for (int k = 0; k < 6; ++k) a[k] = (x[k] - p.in_mean[k]) / p.in_std[k];
  int64_t off = 0;
  for (int l = 0; l < p.n_layers; ++l) {
    const int n_in = p.sizes[l], n_out = p.sizes[l + 1];
    const R* Wl = p.net + off;
    const R* bl = Wl + (int64_t)n_in * n_out;
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
  s[1] = p.sizes[p.n_layers] > 1 ? a[1] : mk_t<T>(R(0));
}

// moments of the five stencil nodes (L, y), (L-1, y), (L-2, y), (L, y-1), (L, y+1)
// from their populations in[9n .. 9n+8]: mac[3n + {0, 1, 2}] = rho - 1, u, v
template <typename T>
__device__ __forceinline__ void stencil_macros(const T* in, T mac[15]) {
#pragma unroll
  for (int n = 0; n < 5; ++n) moments_h(in + 9 * n, mac[3 * n], mac[3 * n + 1], mac[3 * n + 2]);
}

// the six derivatives (p_x, u_x, v_x, p_y, u_y, v_y) of the east node from the
// stencil moments: one-sided second order in x, central in y, p = rho / 3
template <typename T>
__device__ __forceinline__ void features_g(const T mac[15], T fx[6]) {
  using S = typename ScalarOf<T>::type;
  const S cs2 = S(1) / S(3), h = S(0.5);
  fx[0] = h * (S(3) * (cs2 * mac[0]) - S(4) * (cs2 * mac[3]) + cs2 * mac[6]);
  fx[1] = h * (S(3) * mac[1] - S(4) * mac[4] + mac[7]);
  fx[2] = h * (S(3) * mac[2] - S(4) * mac[5] + mac[8]);
  fx[3] = h * (cs2 * mac[12] - cs2 * mac[9]);
  fx[4] = h * (mac[13] - mac[10]);
  fx[5] = h * (mac[14] - mac[11]);
}

// sigma and kappa2 of a node from its features: constants, or the tuner's
// sigma_max sigmoid(s_0) (and kappa2_max sigmoid(s_1) with two outputs)
template <typename T, typename R>
__device__ __forceinline__ void cbc_params_g(const SegParams<R>& p, const T fx[6], T& sigma,
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
// known populations kn = h0(L, y), h1(L-1, y), h2(L, y-1), h4(L, y+1),
// h5(L-1, y-1), h8(L-1, y+1) and the node's sigma, kappa2: Eqs. 20-27, one
// Euler step, Zou & He with the prescribed state, the f_0 correction of Eq. 28
// (or the exact-mass one), then BGK.
template <typename T, typename R>
__device__ void east_core_g(const SegParams<R>& p, const T mac[15], const T kn[6], T sigma,
                            T kappa2, T out[9]) {
  using S = R;
  const S cs2 = S(1) / S(3);
  const S cs = sqrt(cs2);
  const S two_cs2 = S(2) * cs2;
  T fx[6];
  features_g(mac, fx);
  const T px = fx[0], ux = fx[1], vx = fx[2], py = fx[3], vy = fx[5];
  const T dr = mac[0], u0 = mac[1], v0 = mac[2];
  const T rho = S(1) + dr;
  const T pL = cs2 * rho;
  const T L5 = (u0 + cs) * (px + cs * (rho * ux));               // Eq. 22
  const T L3 = u0 * vx;                                          // Eq. 21
  const T T1 = -(v0 * py + pL * vy - cs * (rho * v0 * vy));      // Eq. 23
  const T T3 = -(v0 * vy + py / rho);                            // Eq. 24
  const T T5 = -(v0 * py + pL * vy + cs * (rho * v0 * vy));      // Eq. 25
  const T kappa1 = sigma * p.kfac;                               // Eq. 27
  const T L1 = kappa1 * (cs2 * (dr - p.drho_out)) - kappa2 * T1 + T1;  // Eq. 26
  const T drn = dr + (-(L5 + L1) / two_cs2 + (T5 + T1) / two_cs2);     // Eq. 17
  const T rcs2 = (S(2) * cs) * rho;
  const T un = u0 + (-(L5 - L1) / rcs2 + (T5 - T1) / rcs2);     // Eq. 18
  const T vn = v0 + (-L3 + T3);                                  // Eq. 19
  T g[9];
  g[0] = kn[0];
  g[1] = kn[1];
  g[2] = kn[2];
  g[4] = kn[3];
  g[5] = kn[4];
  g[8] = kn[5];
  T fe[9];
  heq_g(drn, un, vn, fe);
  const T half_t = S(0.5) * ((g[4] - fe[4]) - (g[2] - fe[2]));
  g[3] = fe[3] + (g[1] - fe[1]);
  g[6] = fe[6] + (g[8] - fe[8]) + half_t;
  g[7] = fe[7] + (g[5] - fe[5]) - half_t;
  // rho (1 + u) - (rho0 + 2 rho+) in shifted populations
  const T known = (g[0] + g[2] + g[4]) + S(2) * (g[1] + g[5] + g[8]);
  const T excess = drn + un + drn * un - known;
  if (p.exact) g[0] = g[0] + excess;                             // exact mass
  else g[0] = g[0] + excess / (S(1) + un);                       // Eq. 28
  bgk_h(g, p.omega, out);
}

// offset in a strip state of east input k of node y: k < 45 population k % 9 of
// stencil node k / 9, then the six known pulls
template <typename R>
__device__ __forceinline__ int64_t east_input_offset(const SegParams<R>& p, int y, int k) {
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
template <typename R>
__global__ void seg_init_kernel(const SegParams<R> p) {
  const int s = blockIdx.y;
  const int64_t pl = node_plane(p);
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 9 * pl) return;
  const int j = (int)(k % p.W);
  const int64_t iy = k / p.W;            // i * ny + y
  const int i = (int)(iy / p.ny);
  const double* src = p.bank + (int64_t)p.init_idx[s] * 9 * p.ny * p.bank_w;
  hist_at(p, s, 0)[k] = (R)(src[iy * p.bank_w + (p.bank_w - p.W) + j] - wgt<double>(i));
}

// interior nodes (columns 0 .. W-2): pull and BGK
template <typename R>
__global__ void seg_forward_kernel(const SegParams<R> p, int t) {
  const int s = blockIdx.y;
  const int64_t pl = node_plane(p);
  const int wi = p.W - 1;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p.ny * wi) return;
  const int y = idx / wi, j = idx % wi;
  const R* A = hist_at(p, s, t);
  const R* A0 = hist_at(p, s, 0);
  R* B = hist_at(p, s, t + 1);
  R g[9], out[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int jsrc = j - cx(i);
    const int ysrc = wrap(y - cy(i), p.ny);
    g[i] = jsrc >= 0 ? A[i * pl + (int64_t)ysrc * p.W + jsrc]
                     : A0[i * pl + (int64_t)ysrc * p.W];     // frozen west edge
  }
  bgk_h(g, p.omega, out);
  const int64_t o = (int64_t)y * p.W + j;
#pragma unroll
  for (int i = 0; i < 9; ++i) B[i * pl + o] = out[i];
}

// east nodes (column W-1): the characteristic outflow with the tuner
template <typename R>
__global__ void seg_forward_east_kernel(const SegParams<R> p, int t) {
  const int s = blockIdx.y;
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= p.ny) return;
  const int64_t pl = node_plane(p);
  const R* A = hist_at(p, s, t);
  R* B = hist_at(p, s, t + 1);
  R in[kEastInputs], mac[15], fx[6], sigma, kappa2, out[9];
  for (int k = 0; k < kEastInputs; ++k) in[k] = A[east_input_offset(p, y, k)];
  stencil_macros(in, mac);
  features_g(mac, fx);
  cbc_params_g(p, fx, sigma, kappa2);
  east_core_g(p, mac, in + 45, sigma, kappa2, out);
  const int64_t o = (int64_t)y * p.W + p.W - 1;
#pragma unroll
  for (int i = 0; i < 9; ++i) B[i * pl + o] = out[i];
}

// loss of the batch (mean over segments, FP64) and lambda at t = n_t
template <typename R>
__global__ void __launch_bounds__(128) seg_loss_kernel(const SegParams<R> p) {
  __shared__ double red[128];
  const int s = blockIdx.y;
  const int64_t pl = node_plane(p);
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  double contrib = 0.0;
  if (idx < pl) {
    const int y = idx / p.W, j = idx % p.W;
    double lam[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (j >= p.W - p.n_t) {
      const R* A = hist_at(p, s, p.n_t);
      const double* Rf = p.bank + (int64_t)p.final_idx[s] * 9 * p.ny * p.bank_w;
      double dr = 0.0, jx = 0.0, jy = 0.0, rr = 0.0, jxr = 0.0, jyr = 0.0;
      for (int i = 0; i < 9; ++i) {
        const double h = (double)A[i * pl + idx];
        const double fr = Rf[((int64_t)i * p.ny + y) * p.bank_w + (p.bank_w - p.W) + j];
        dr += h;
        jx += cx(i) * h;
        jy += cy(i) * h;
        rr += fr;
        jxr += cx(i) * fr;
        jyr += cy(i) * fr;
      }
      const double rho = 1.0 + dr, u = jx / rho, v = jy / rho;
      const double ur = jxr / rr, vr = jyr / rr;
      const double n = (double)p.n_t * p.ny;
      const double scale = 1.0 / p.n_seg;
      const double d_r = rho - rr, du = u - ur, dv = v - vr;
      contrib = scale * (d_r * d_r / n + (du * du + dv * dv) / (2.0 * n));
      for (int i = 0; i < 9; ++i)
        lam[i] = scale * (2.0 * d_r / n + (du * (cx(i) - u) + dv * (cy(i) - v)) / (n * rho));
    }
    for (int i = 0; i < 9; ++i) p.lam_in[(int64_t)s * 9 * pl + i * pl + idx] = (R)lam[i];
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
template <typename R>
__global__ void seg_adj_interior_kernel(const SegParams<R> p, int t) {
  const int s = blockIdx.y;
  const int64_t pl = node_plane(p);
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= pl) return;
  const int y = idx / p.W, j = idx % p.W;
  if (j == p.W - 1) return;
  const R* A = hist_at(p, s, t);
  const R* A0 = hist_at(p, s, 0);
  const R* lam = p.lam_in + (int64_t)s * 9 * pl;
  R g[9], l[9];
  bool any = false;
  for (int i = 0; i < 9; ++i) {
    l[i] = lam[i * pl + idx];
    any |= l[i] != R(0);
  }
  R* mu = p.mu + (int64_t)s * 9 * pl;
  if (!any) {
    for (int i = 0; i < 9; ++i) mu[i * pl + idx] = R(0);
    return;
  }
  for (int i = 0; i < 9; ++i) {
    const int jsrc = j - cx(i);
    const int ysrc = wrap(y - cy(i), p.ny);
    g[i] = jsrc >= 0 ? A[i * pl + (int64_t)ysrc * p.W + jsrc] : A0[i * pl + (int64_t)ysrc * p.W];
  }
  R dr, u, v;
  moments_h(g, dr, u, v);
  // out_k = h_k - omega (h_k - heq_k); heq_k + w_k = w_k rho (1 + a_k),
  // a_k = 3 cu + 4.5 cu^2 - 1.5 |u|^2; d rho / dh_i = 1, du / dh_i = (c_ix - u) / rho
  R sr = 0, su = 0, sv = 0;
  const R usq = u * u + v * v;
  for (int k = 0; k < 9; ++k) {
    const R cu = R(cx(k)) * u + R(cy(k)) * v;
    const R wl = wgt<R>(k) * l[k];
    sr += wl * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * usq);
    su += wl * (R(3 * cx(k)) + R(9) * cu * R(cx(k)) - R(3) * u);
    sv += wl * (R(3 * cy(k)) + R(9) * cu * R(cy(k)) - R(3) * v);
  }
  const R om = p.omega;
  for (int i = 0; i < 9; ++i)
    mu[i * pl + idx] = (R(1) - om) * l[i] + om * (sr + su * (R(cx(i)) - u) + sv * (R(cy(i)) - v));
}

// Input adjoints of lambda_{t+1}(L, y) . east_node, one warp per east node:
// lanes 0..5 differentiate the tuner along each feature (its Jacobian, once);
// lanes 0..22 differentiate the core along the 15 stencil moments, the 6 known
// pulls, sigma and kappa2 (forward mode); the moments' adjoints take the
// feature path (the features are linear in the moments) and become population
// adjoints through d(rho, u, v)/dh.  Records (features, dL/dsigma, dL/dkappa2)
// feed the parameter gradient.
template <typename R>
__global__ void __launch_bounds__(32 * kAdjWarps) seg_adj_east_kernel(const SegParams<R> p, int t) {
  using D = DualT<R>;
  __shared__ R sh[kAdjWarps][kAdjShared];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.y;
  const int y = blockIdx.x * kAdjWarps + warp;
  if (y >= p.ny) return;                     // whole warps only
  R* in = sh[warp];
  R* mac = in + 51;
  R* lam = mac + 15;
  R* fx = lam + 9;
  R* gs = fx + 6;
  R* gk = gs + 6;
  R* sk = gk + 6;
  R* a = sk + 2;
  R* mb = a + 23;
  const int64_t pl = node_plane(p);
  const R* A = hist_at(p, s, t);
  for (int k = lane; k < kEastInputs; k += 32) in[k] = A[east_input_offset(p, y, k)];
  if (lane < 9) lam[lane] = p.lam_in[(int64_t)s * 9 * pl + lane * pl + (int64_t)y * p.W + p.W - 1];
  __syncwarp();
  if (lane < 5) {
    R r, u, v;
    moments_h(in + 9 * lane, r, u, v);
    mac[3 * lane] = r;
    mac[3 * lane + 1] = u;
    mac[3 * lane + 2] = v;
  }
  __syncwarp();
  if (lane == 0) features_g(mac, fx);
  __syncwarp();
  if (lane < 6) {
    D xf[6];
    for (int k = 0; k < 6; ++k) xf[k] = {fx[k], k == lane ? R(1) : R(0)};
    D sg, kp;
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
    D m[15], kn[6];
    for (int q = 0; q < 15; ++q) m[q] = {mac[q], q == lane ? R(1) : R(0)};
    for (int q = 0; q < 6; ++q) kn[q] = {in[45 + q], 15 + q == lane ? R(1) : R(0)};
    const D sg = {sk[0], lane == 21 ? R(1) : R(0)};
    const D kp = {sk[1], lane == 22 ? R(1) : R(0)};
    D out[9];
    east_core_g(p, m, kn, sg, kp, out);
    R acc = 0;
    for (int i = 0; i < 9; ++i) acc += lam[i] * out[i].d;
    a[lane] = acc;
  }
  __syncwarp();
  if (lane < 15) {
    // feature path: fbar_f = dL/dsigma dsigma/dfx_f + dL/dkappa2 dkappa2/dfx_f,
    // times d fx_f / d mac_lane (the linear feature map, by one dual pass)
    D md[15], fd[6];
    for (int q = 0; q < 15; ++q) md[q] = {mac[q], q == lane ? R(1) : R(0)};
    features_g(md, fd);
    R acc = a[lane];
    for (int f = 0; f < 6; ++f) acc += (a[21] * gs[f] + a[22] * gk[f]) * fd[f].d;
    mb[lane] = acc;
  }
  __syncwarp();
  R* e = p.east + ((int64_t)s * p.ny + y) * kEastInputs;
  for (int k = lane; k < kEastInputs; k += 32) {
    R v;
    if (k < 45) {
      const int n = k / 9, i = k % 9;
      const R rho = R(1) + mac[3 * n], uu = mac[3 * n + 1], vv = mac[3 * n + 2];
      v = mb[3 * n] + (mb[3 * n + 1] * (R(cx(i)) - uu) + mb[3 * n + 2] * (R(cy(i)) - vv)) / rho;
    } else {
      v = a[15 + (k - 45)];
    }
    e[k] = v;
  }
  if (lane == 0) {
    R* rec = p.rec + (((int64_t)s * p.n_t + t) * p.ny + y) * kRecWidth;
    for (int k = 0; k < 6; ++k) rec[k] = fx[k];
    rec[6] = a[21];
    rec[7] = a[22];
  }
}

// lambda_t from the consumers' mu and the east nodes' input adjoints
template <typename R>
__global__ void seg_gather_kernel(const SegParams<R> p) {
  const int s = blockIdx.y;
  const int64_t pl = node_plane(p);
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= pl) return;
  const int y = idx / p.W, j = idx % p.W, W = p.W, ny = p.ny;
  const R* mu = p.mu + (int64_t)s * 9 * pl;
  const R* E = p.east + (int64_t)s * ny * kEastInputs;
  R* lam = p.lam_out + (int64_t)s * 9 * pl;
  const int yu = wrap(y + 1, ny), yd = wrap(y - 1, ny);
  for (int i = 0; i < 9; ++i) {
    R acc = 0;
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
// through the tuner in R; each chunk's per-parameter sum (records in order) is
// added to the block's FP64 accumulator; one partial per block
template <typename R>
struct GradParams {
  int n_layers, sizes[LBM_MLP_MAX_LAYERS + 1], act, n_out;
  const R* net;
  const R* in_mean;
  const R* in_std;
  R sig_max, kap;
  int64_t n_params, n_rec;
  const R* rec;
  double* partial;       // [gridDim.x][n_params]
  int in_off[LBM_MLP_MAX_LAYERS], dl_off[LBM_MLP_MAX_LAYERS], per_rec;
};

template <typename R>
__global__ void __launch_bounds__(kGradThreads) tuner_grad_kernel(const GradParams<R> q) {
  extern __shared__ double sm[];
  double* gacc = sm;                                          // [n_params]
  R* buf = reinterpret_cast<R*>(sm + ((q.n_params + 1) & ~int64_t(1)));  // [kGradChunk][per_rec]
  for (int64_t k = threadIdx.x; k < q.n_params; k += blockDim.x) gacc[k] = 0.0;
  const int64_t chunks = (q.n_rec + kGradChunk - 1) / kGradChunk;
  int64_t offs[LBM_MLP_MAX_LAYERS];
  {
    int64_t o2 = 0;
    for (int l = 0; l < q.n_layers; ++l) {
      offs[l] = o2;
      o2 += (int64_t)q.sizes[l] * q.sizes[l + 1] + q.sizes[l + 1];
    }
  }
  for (int64_t c = blockIdx.x; c < chunks; c += gridDim.x) {
    const int64_t r0 = c * kGradChunk;
    const int64_t left = q.n_rec - r0;
    const int nr = left < kGradChunk ? (int)left : kGradChunk;
    __syncthreads();
    if ((int)threadIdx.x < nr) {
      const R* rc = q.rec + (r0 + threadIdx.x) * kRecWidth;
      R* mine = buf + threadIdx.x * q.per_rec;
      R a[kSegMaxW], z[LBM_MLP_MAX_LAYERS][kSegMaxW];
      for (int k = 0; k < 6; ++k) a[k] = (rc[k] - q.in_mean[k]) / q.in_std[k];
      for (int l = 0; l < q.n_layers; ++l) {
        const int n_in = q.sizes[l], n_out = q.sizes[l + 1];
        const R* Wl = q.net + offs[l];
        const R* bl = Wl + (int64_t)n_in * n_out;
        for (int k = 0; k < n_in; ++k) mine[q.in_off[l] + k] = a[k];
        R b[kSegMaxW];
        for (int j = 0; j < n_out; ++j) {
          R acc = bl[j];
          for (int k = 0; k < n_in; ++k) acc = acc + Wl[j * n_in + k] * a[k];
          z[l][j] = acc;
          b[j] = l == q.n_layers - 1 ? acc : act_g(acc, q.act);
        }
        for (int j = 0; j < n_out; ++j) a[j] = b[j];
      }
      // output deltas: sigma = sig_max sigmoid(s0), kappa2 = kap sigmoid(s1)
      R dl[kSegMaxW];
      {
        const R s0 = sigmoid_g(a[0]);
        dl[0] = rc[6] * q.sig_max * s0 * (R(1) - s0);
        if (q.n_out > 1) {
          const R s1 = sigmoid_g(a[1]);
          dl[1] = rc[7] * q.kap * s1 * (R(1) - s1);
        }
      }
      for (int l = q.n_layers - 1; l >= 0; --l) {
        const int n_in = q.sizes[l], n_out = q.sizes[l + 1];
        for (int j = 0; j < n_out; ++j) mine[q.dl_off[l] + j] = dl[j];
        if (l == 0) break;
        const R* Wl = q.net + offs[l];
        R nd[kSegMaxW];
        for (int k = 0; k < n_in; ++k) {
          R acc = 0;
          for (int j = 0; j < n_out; ++j) acc += Wl[j * n_in + k] * dl[j];
          const R zz = z[l - 1][k];
          R dz;
          if (q.act == 0) {
            const R th = tanh_s(zz);
            dz = R(1) - th * th;
          } else {
            dz = zz > R(0) ? R(1) : R(0.01);
          }
          nd[k] = acc * dz;
        }
        for (int k = 0; k < n_in; ++k) dl[k] = nd[k];
      }
    }
    __syncthreads();
    // parameter sums over this chunk's records, in record order
    for (int l = 0; l < q.n_layers; ++l) {
      const int n_in = q.sizes[l], n_out = q.sizes[l + 1];
      const int64_t nw = (int64_t)n_in * n_out;
      for (int64_t k = threadIdx.x; k < nw + n_out; k += blockDim.x) {
        R acc = 0;
        if (k < nw) {
          const int j = (int)(k / n_in), kk = (int)(k % n_in);
          for (int r = 0; r < nr; ++r) {
            const R* m = buf + r * q.per_rec;
            acc += m[q.dl_off[l] + j] * m[q.in_off[l] + kk];
          }
        } else {
          const int j = (int)(k - nw);
          for (int r = 0; r < nr; ++r) acc += buf[r * q.per_rec + q.dl_off[l] + j];
        }
        gacc[offs[l] + k] += (double)acc;
      }
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

// Adam (Kingma & Ba 2015) in FP64; c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t);
// prm_r receives the parameters in the compute type
template <typename R>
__global__ void adam_kernel(double* prm, R* prm_r, double* m, double* v, const double* g,
                            int64_t n, double lr, double b1, double b2, double eps, double c1,
                            double c2) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  m[k] = b1 * m[k] + (1.0 - b1) * g[k];
  v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k];
  const double mh = m[k] * c1, vh = v[k] * c2;
  const double np = prm[k] - lr * mh / (sqrt(vh) + eps);
  prm[k] = np;
  prm_r[k] = (R)np;
}

template <typename R>
__global__ void to_compute_kernel(const double* src, R* dst, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) dst[k] = (R)src[k];
}

// Mean and population standard deviation of the six tuner features over the
// east nodes of every bank state (FP64, one block, fixed summation order).
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
        for (int i = 0; i < 9; ++i)
          in[9 * q + i] = A[((int64_t)i * ny + ys[q]) * bank_w + js[q]] - wgt<double>(i);
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
      if (pass == 0) {
        mean[threadIdx.x] = m;
        out[threadIdx.x] = m;
      } else {
        out[6 + threadIdx.x] = sqrt(m);
      }
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

// Device scratch of one call, from the process-wide default allocator
// (lbm_set_default_allocator), freed when the call returns.
struct Scratch {
  std::vector<void*> ptrs;
  lbm_allocator a{};
  bool have = default_allocator(&a);
  ~Scratch() {
    // an injected allocator may hand the memory out again at once: on an
    // early exit kernels of this call could still be using it
    if (have && !ptrs.empty()) cudaDeviceSynchronize();
    for (void* q : ptrs) dev_free_raw(have ? &a : nullptr, q);
  }
  template <typename T>
  T* get(size_t n) {
    void* q = dev_alloc_raw(have ? &a : nullptr, std::max<size_t>(n * sizeof(T), 16));
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
  if (g->precision != LBM_FP64 && g->precision != LBM_FP32)
    return seg_fail(LBM_ERR_ARG, "precision must be LBM_FP64 or LBM_FP32");
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

// Loss + gradient evaluations of batches of segments.  net64() holds the FP64
// parameters; load_params() refreshes the compute-type copy from it.
class SegmentRunnerBase {
 public:
  virtual ~SegmentRunnerBase() = default;
  virtual double* net64() = 0;
  virtual void load_params() = 0;
  virtual int* init_idx() = 0;
  virtual int* final_idx() = 0;
  virtual void run(int n, double* d_grad, double* d_loss) = 0;
  virtual void adam(double* m, double* v, const double* g, double lr, double b1, double b2,
                    double eps, double c1, double c2) = 0;
};

template <typename R>
class SegmentRunner : public SegmentRunnerBase {
 public:
  SegmentRunner(const lbm_cbc_segments* g, const lbm_mlp* tuner, int64_t np, int max_batch,
                cudaStream_t st)
      : st_(st), np_(np) {
    p_ = SegParams<R>{};
    p_.ny = g->ny;
    p_.n_t = g->n_t;
    p_.W = std::max(2 * g->n_t, 3);
    p_.bank_w = g->bank_width;
    p_.omega = (R)(1.0 / g->tau);
    p_.drho_out = (R)(g->rho_out - 1.0);
    p_.sig_max = (R)g->sigma;
    p_.kap = (R)g->kappa2;
    const double cs = std::sqrt(1.0 / 3.0);
    const double length = g->length > 0.0 ? g->length : (double)g->nx;
    p_.kfac = (R)((1.0 - g->mach * g->mach) * cs / length);
    p_.exact = g->exact_mass ? 1 : 0;
    p_.n_layers = tuner->n_layers;
    for (int l = 0; l <= LBM_MLP_MAX_LAYERS; ++l)
      p_.sizes[l] = l <= tuner->n_layers ? tuner->sizes[l] : 0;
    p_.act = tuner->act;
    p_.bank = g->bank;
    const int64_t pl = (int64_t)p_.ny * p_.W;
    d_net64_ = sc_.get<double>(np);
    d_net_ = sc_.get<R>(np);
    d_norm_ = sc_.get<R>(12);
    std::vector<R> norm(12);
    for (int k = 0; k < 6; ++k) {
      norm[k] = tuner->in_mean ? (R)tuner->in_mean[k] : R(0);
      norm[6 + k] = tuner->in_std ? (R)tuner->in_std[k] : R(1);
    }
    ck(cudaMemcpyAsync(d_norm_, norm.data(), 12 * sizeof(R), cudaMemcpyHostToDevice, st_), "copy");
    ck(cudaStreamSynchronize(st_), "sync");
    p_.net = d_net_;
    p_.in_mean = d_norm_;
    p_.in_std = d_norm_ + 6;
    p_.init_idx = d_init_ = sc_.get<int>(max_batch);
    p_.final_idx = d_final_ = sc_.get<int>(max_batch);
    p_.hist = sc_.get<R>((size_t)max_batch * (p_.n_t + 1) * 9 * pl);
    p_.lam_in = sc_.get<R>((size_t)max_batch * 9 * pl);
    p_.lam_out = sc_.get<R>((size_t)max_batch * 9 * pl);
    p_.mu = sc_.get<R>((size_t)max_batch * 9 * pl);
    p_.east = sc_.get<R>((size_t)max_batch * p_.ny * kEastInputs);
    p_.rec = sc_.get<R>((size_t)max_batch * p_.n_t * p_.ny * kRecWidth);
    loss_blocks_ = (int)((pl + 127) / 128);
    p_.loss_part = sc_.get<double>((size_t)max_batch * loss_blocks_);
    grad_part_ = sc_.get<double>((size_t)kGradBlocks * np);
    // gradient kernel layout: per record the inputs of every layer, then the deltas
    gq_ = GradParams<R>{};
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
    grad_smem_ = (size_t)((np + 1) & ~int64_t(1)) * sizeof(double) +
                 (size_t)kGradChunk * o * sizeof(R);
    ck(cudaFuncSetAttribute(tuner_grad_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)grad_smem_), "smem attribute");
  }

  double* net64() override { return d_net64_; }
  int* init_idx() override { return d_init_; }
  int* final_idx() override { return d_final_; }

  void load_params() override {
    to_compute_kernel<R><<<(unsigned)((np_ + 127) / 128), 128, 0, st_>>>(d_net64_, d_net_, np_);
    ck(cudaGetLastError(), "parameter copy");
  }

  void adam(double* m, double* v, const double* g, double lr, double b1, double b2, double eps,
            double c1, double c2) override {
    adam_kernel<R><<<(unsigned)((np_ + 127) / 128), 128, 0, st_>>>(d_net64_, d_net_, m, v, g, np_,
                                                                  lr, b1, b2, eps, c1, c2);
    ck(cudaGetLastError(), "adam launch");
  }

  void run(int n, double* d_grad, double* d_loss) override {
    SegParams<R> p = p_;
    p.n_seg = n;
    const int64_t pl = (int64_t)p.ny * p.W;
    const dim3 gn((unsigned)((pl + 127) / 128), (unsigned)n);
    const dim3 gi((unsigned)((9 * pl + 127) / 128), (unsigned)n);
    const dim3 gf((unsigned)((p.ny * (p.W - 1) + 127) / 128), (unsigned)n);
    const dim3 ge((unsigned)((p.ny + 63) / 64), (unsigned)n);
    const dim3 ga((unsigned)((p.ny + kAdjWarps - 1) / kAdjWarps), (unsigned)n);
    seg_init_kernel<R><<<gi, 128, 0, st_>>>(p);
    for (int t = 0; t < p.n_t; ++t) {
      seg_forward_kernel<R><<<gf, 128, 0, st_>>>(p, t);
      seg_forward_east_kernel<R><<<ge, 64, 0, st_>>>(p, t);
    }
    seg_loss_kernel<R><<<gn, 128, 0, st_>>>(p);
    sum_loss_kernel<<<1, 32, 0, st_>>>(p.loss_part, (int64_t)n * loss_blocks_, d_loss);
    for (int t = p.n_t - 1; t >= 0; --t) {
      seg_adj_interior_kernel<R><<<gn, 128, 0, st_>>>(p, t);
      seg_adj_east_kernel<R><<<ga, 32 * kAdjWarps, 0, st_>>>(p, t);
      if (t > 0) {
        seg_gather_kernel<R><<<gn, 128, 0, st_>>>(p);
        std::swap(p.lam_in, p.lam_out);
      }
    }
    GradParams<R> q = gq_;
    q.net = d_net_;
    q.in_mean = d_norm_;
    q.in_std = d_norm_ + 6;
    q.n_rec = (int64_t)n * p.n_t * p.ny;
    q.rec = p.rec;
    q.partial = grad_part_;
    tuner_grad_kernel<R><<<kGradBlocks, kGradThreads, grad_smem_, st_>>>(q);
    sum_partials_kernel<<<(unsigned)((q.n_params + 127) / 128), 128, 0, st_>>>(
        grad_part_, kGradBlocks, q.n_params, d_grad);
    ck(cudaGetLastError(), "segment launches");
  }

 private:
  cudaStream_t st_;
  int64_t np_;
  Scratch sc_;
  SegParams<R> p_;
  GradParams<R> gq_;
  double* d_net64_ = nullptr;
  R* d_net_ = nullptr;
  R* d_norm_ = nullptr;
  int* d_init_ = nullptr;
  int* d_final_ = nullptr;
  double* grad_part_ = nullptr;
  int loss_blocks_ = 0;
  size_t grad_smem_ = 0;
};

SegmentRunnerBase* make_runner(const lbm_cbc_segments* g, const lbm_mlp* tuner, int64_t np,
                               int max_batch, cudaStream_t st) {
  if (g->precision == LBM_FP32) return new SegmentRunner<float>(g, tuner, np, max_batch, st);
  return new SegmentRunner<double>(g, tuner, np, max_batch, st);
}

lbm_status check_indices(const lbm_cbc_segments* g) {
  if (g->n_seg < 1 || g->n_seg > 65535 || !g->init_state || !g->final_state)
    return seg_fail(LBM_ERR_ARG, "n_seg in [1, 65535] and the index arrays are required");
  for (int k = 0; k < g->n_seg; ++k)
    if (g->init_state[k] < 0 || g->init_state[k] >= g->n_states || g->final_state[k] < 0 ||
        g->final_state[k] >= g->n_states)
      return seg_fail(LBM_ERR_ARG, "state index out of range");
  return LBM_OK;
}

lbm_status cuda_fail(const CudaError& ce) {
  set_last_error(std::string(ce.what) + ": " + cudaGetErrorString(ce.e));
  return ce.e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

}  // namespace
}  // namespace lbm

extern "C" {

lbm_status lbm_copy_columns(lbm_sim* s, int32_t x0, int32_t width, double* dev_out) {
  using namespace lbm;
  if (!s || !s->buf[0]) return seg_fail(LBM_ERR_STATE, "sim is not initialised");
  if (!dev_out) return seg_fail(LBM_ERR_ARG, "dev_out is NULL");
  if (s->layout == LBM_LAYOUT_AA)
    return seg_fail(LBM_ERR_UNSUPPORTED, "column copies need the two-buffer (AB) layout");
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
    return cuda_fail(ce);
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
    return cuda_fail(ce);
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
    std::unique_ptr<SegmentRunnerBase> run(make_runner(g, tuner, np, g->n_seg, st));
    Scratch sc;
    double* d_grad = sc.get<double>(np);
    double* d_loss = sc.get<double>(1);
    ck(cudaMemcpyAsync(run->net64(), params, np * 8, cudaMemcpyHostToDevice, st), "copy");
    run->load_params();
    ck(cudaMemcpyAsync(run->init_idx(), g->init_state, g->n_seg * 4, cudaMemcpyHostToDevice, st),
       "copy");
    ck(cudaMemcpyAsync(run->final_idx(), g->final_state, g->n_seg * 4, cudaMemcpyHostToDevice, st),
       "copy");
    run->run(g->n_seg, d_grad, d_loss);
    ck(cudaMemcpyAsync(loss, d_loss, 8, cudaMemcpyDeviceToHost, st), "copy");
    if (grad) ck(cudaMemcpyAsync(grad, d_grad, np * 8, cudaMemcpyDeviceToHost, st), "copy");
    ck(cudaStreamSynchronize(st), "sync");
  } catch (const CudaError& ce) {
    return cuda_fail(ce);
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
    std::unique_ptr<SegmentRunnerBase> run(make_runner(g, tuner, np, batch, st));
    Scratch sc;
    double* d_grad = sc.get<double>(np);
    double* d_m = sc.get<double>(np);
    double* d_v = sc.get<double>(np);
    double* d_loss = sc.get<double>(n_steps);
    ck(cudaMemcpyAsync(run->net64(), params, np * 8, cudaMemcpyHostToDevice, st), "copy");
    run->load_params();
    if (adam_m) ck(cudaMemcpyAsync(d_m, adam_m, np * 8, cudaMemcpyHostToDevice, st), "copy");
    else ck(cudaMemsetAsync(d_m, 0, np * 8, st), "memset");
    if (adam_v) ck(cudaMemcpyAsync(d_v, adam_v, np * 8, cudaMemcpyHostToDevice, st), "copy");
    else ck(cudaMemsetAsync(d_v, 0, np * 8, st), "memset");
    // the bank indices of every step's batch, gathered on the host (small)
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
      ck(cudaMemcpyAsync(run->init_idx(), d_bi + k * batch, batch * 4, cudaMemcpyDeviceToDevice,
                         st), "copy");
      ck(cudaMemcpyAsync(run->final_idx(), d_bf + k * batch, batch * 4, cudaMemcpyDeviceToDevice,
                         st), "copy");
      run->run(batch, d_grad, d_loss + k);
      const double tt = (double)(o->adam_t0 + k + 1);
      const double c1 = 1.0 / (1.0 - std::pow(o->beta1, tt));
      const double c2 = 1.0 / (1.0 - std::pow(o->beta2, tt));
      run->adam(d_m, d_v, d_grad, o->lr, o->beta1, o->beta2, o->eps, c1, c2);
    }
    ck(cudaMemcpyAsync(params, run->net64(), np * 8, cudaMemcpyDeviceToHost, st), "copy");
    if (adam_m) ck(cudaMemcpyAsync(adam_m, d_m, np * 8, cudaMemcpyDeviceToHost, st), "copy");
    if (adam_v) ck(cudaMemcpyAsync(adam_v, d_v, np * 8, cudaMemcpyDeviceToHost, st), "copy");
    if (loss_log) ck(cudaMemcpyAsync(loss_log, d_loss, n_steps * 8, cudaMemcpyDeviceToHost, st), "copy");
    ck(cudaStreamSynchronize(st), "sync");
  } catch (const CudaError& ce) {
    return cuda_fail(ce);
  }
  return LBM_OK;
}

}  // extern "C"
