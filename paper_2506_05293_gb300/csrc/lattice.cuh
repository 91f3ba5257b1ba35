// D2Q9 lattice, shifted-population equilibrium and collision operators for the
// GB300 kernels.
//
// Populations are stored shifted: h_i = f_i - w_i (Sec. 2.1, Eqs. 2-4 are
// linear in f apart from the equilibrium, and the lattice weights are the rest
// state).  Storing the small deviation instead of f keeps FP32 and FP16 storage
// accurate: the rest weights never pass through a rounding.
//
// Velocity numbering (Sec. 2.2: unknowns 3, 6, 7 on the east side,
// rho+ = f1 + f5 + f8, rho0 = f0 + f2 + f4):
//   c0=(0,0) c1=(1,0) c2=(0,1) c3=(-1,0) c4=(0,-1)
//   c5=(1,1) c6=(-1,1) c7=(-1,-1) c8=(1,-1)
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

namespace lbm {

__host__ __device__ constexpr int cx(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) {
  return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5);
}
template <typename R>
__host__ __device__ constexpr R wgt(int i) {
  return i == 0 ? R(4) / R(9) : (i <= 4 ? R(1) / R(9) : R(1) / R(36));
}

static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2, "opp");
static_assert(opp(5) == 7 && opp(6) == 8 && opp(7) == 5 && opp(8) == 6, "opp");

// ---- storage <-> compute conversions -------------------------------------
template <typename S> struct Compute { using R = float; };
template <> struct Compute<double> { using R = double; };

template <typename R> __device__ __forceinline__ R to_r(double v) { return (R)v; }
template <typename R> __device__ __forceinline__ R to_r(float v) { return (R)v; }
template <typename R> __device__ __forceinline__ R to_r(__half v) { return (R)__half2float(v); }

template <typename S> __device__ __forceinline__ S from_r(double v) { return (S)v; }
template <typename S> __device__ __forceinline__ S from_r(float v) { return (S)v; }
template <> __device__ __forceinline__ __half from_r<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __half from_r<__half>(double v) { return __float2half_rn((float)v); }

// ---- equilibrium in shifted form ----------------------------------------
// f^eq_i - w_i = w_i (drho + rho (3 c.u + 9/2 (c.u)^2 - 3/2 u.u)), Eq. 3 with
// c_s^2 = 1/3 and rho = 1 + drho.
template <typename R>
__device__ __forceinline__ void heq_all(R drho, R ux, R uy, R heq[9]) {
  const R rho = R(1) + drho;
  const R usq15 = R(1.5) * (ux * ux + uy * uy);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const R cu = R(cx(i)) * ux + R(cy(i)) * uy;
    heq[i] = wgt<R>(i) * (drho + rho * (R(3) * cu + R(4.5) * cu * cu - usq15));
  }
}

// ---- explicitly rounded arithmetic -------------------------------------------
// The collision is written once over its arithmetic type V (float or double)
// with every operation rounding once and none contracted by the compiler, so
// every kernel that collides a node -- staged, register, in-place, boundary
// blocks -- gets the same bits for it.
template <typename V> struct Ar;
template <> struct Ar<float> {
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
  using T = float;                                  // component type
  static __device__ __forceinline__ float lit(double v) { return (float)v; }   // exact constants
  static __device__ __forceinline__ float splat(float v) { return v; }
  static __device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }   // correctly rounded
  static __device__ __forceinline__ bool bad(float x) { return !(fabsf(x) < 1e30f); }
};
template <> struct Ar<double> {
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
  using T = double;
  static __device__ __forceinline__ double lit(double v) { return v; }
  static __device__ __forceinline__ double splat(double v) { return v; }
  static __device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }
  static __device__ __forceinline__ bool bad(double x) { return !(fabs(x) < 1e30); }
};

// The same equilibrium evaluated pairwise: for a direction i and its opposite
// ibar, c.u changes sign, so h^eq_i,ibar = s_i +- a_i with
// s_i = w_i (drho - 3/2 rho u.u + 9/2 rho (c_i.u)^2) and a_i = 3 w_i rho c_i.u.
template <typename V>
__device__ __forceinline__ void heq_sym(V drho, V ux, V uy, V heq[9]) {
  using A = Ar<V>;
  const V rho = A::add(A::lit(1), drho);
  const V usq = A::fma(ux, ux, A::mul(uy, uy));
  const V base = A::fma(A::mul(A::lit(-1.5), rho), usq, drho);        // drho - 3/2 rho u.u
  const V r45 = A::mul(A::lit(4.5), rho), r3 = A::mul(A::lit(3), rho);
  heq[0] = A::mul(A::splat(wgt<typename A::T>(0)), base);
  // direction pair (i, ibar) along the component cu = c_i.u
  auto pair = [&](int i, int ib, V cu) {
    const V w = A::splat(wgt<typename A::T>(i));
    const V s = A::mul(w, A::fma(A::mul(r45, cu), cu, base));
    const V a = A::mul(A::mul(w, r3), cu);
    heq[i] = A::add(s, a);
    heq[ib] = A::sub(s, a);
  };
  pair(1, 3, ux);
  pair(2, 4, uy);
  pair(5, 7, A::add(ux, uy));   // c5 = (1, 1); c7 = -c5
  pair(6, 8, A::sub(uy, ux));   // c6 = (-1, 1); c8 = -c6
}

// rho - 1 and momentum of shifted populations (sum w_i = 1, sum w_i c_i = 0)
template <typename V>
__device__ __forceinline__ void moments_shifted(const V h[9], V& drho, V& jx, V& jy) {
  using A = Ar<V>;
  drho = A::add(A::add(A::add(A::add(h[0], h[2]), A::add(h[4], h[1])),
                       A::add(A::add(h[3], h[5]), A::add(h[6], h[7]))),
                h[8]);
  jx = A::add(A::add(A::sub(h[1], h[3]), A::sub(h[5], h[6])), A::sub(h[8], h[7]));
  jy = A::sub(A::add(A::sub(h[2], h[4]), A::add(h[5], h[6])), A::add(h[7], h[8]));
}

// ---- collision operators -------------------------------------------------
// BGK (Eq. 2): h* = h - omega (h - h^eq), omega = 1 / tau.
template <typename V>
__device__ __forceinline__ void collide_bgk(V h[9], V omega, V& drho_out, V& ux_out, V& uy_out) {
  using A = Ar<V>;
  V drho, jx, jy;
  moments_shifted(h, drho, jx, jy);
  const V inv_rho = A::rcp(A::add(A::lit(1), drho));
  const V ux = A::mul(jx, inv_rho), uy = A::mul(jy, inv_rho);
  V heq[9];
  heq_sym(drho, ux, uy, heq);
  const V nomega = A::mul(A::lit(-1), omega);
#pragma unroll
  for (int i = 0; i < 9; ++i) h[i] = A::fma(nomega, A::sub(h[i], heq[i]), h[i]);
  drho_out = drho; ux_out = ux; uy_out = uy;
}

// MRT with Lallemand & Luo's orthogonal basis (rho, e, eps, jx, qx, jy, qy,
// pxx, pxy).  Only the six non-conserved moments of the non-equilibrium part
// n = h - h^eq relax, each at its own rate: h* = h - M^-1 S M n, and
// M^-1 = M^T diag(1 / |row_k|^2) with |row|^2 = (9, 36, 36, 6, 12, 6, 12, 4, 4).
template <typename R>
struct MrtRates { R se, seps, sqx, sqy, snxx, snxy; };

template <typename V, typename R>
__device__ __forceinline__ void collide_mrt(V h[9], const MrtRates<R>& s, V& drho_out, V& ux_out,
                                            V& uy_out) {
  using A = Ar<V>;
  V drho, jx, jy;
  moments_shifted(h, drho, jx, jy);
  const V rho = A::add(A::lit(1), drho);
  const V inv_rho = A::rcp(rho);
  const V ux = A::mul(jx, inv_rho), uy = A::mul(jy, inv_rho);
  // the six non-conserved moments of h (rows of M written out; integer
  // coefficients; q(h) = j - 3 (h_1 - h_3) and its y twin) minus those of the
  // shifted equilibrium: e = -2 drho + 3 rho u.u, eps = drho - 3 rho u.u,
  // q = -j, pxx = rho (ux^2 - uy^2), pxy = rho ux uy -- the moments of
  // n = h - h^eq without forming h^eq
  const V axis = A::add(A::add(h[1], h[2]), A::add(h[3], h[4]));
  const V diag = A::add(A::add(h[5], h[6]), A::add(h[7], h[8]));
  const V two = A::lit(2);
  const V ru2 = A::mul(rho, A::fma(ux, ux, A::mul(uy, uy)));
  const V m_e = A::sub(A::fma(two, diag, A::sub(A::mul(A::lit(-4), h[0]), axis)),
                       A::fma(A::lit(3), ru2, A::mul(A::lit(-2), drho)));
  const V m_eps = A::sub(A::add(A::fma(A::lit(-2), axis, A::mul(A::lit(4), h[0])), diag),
                         A::fma(A::lit(-3), ru2, drho));
  const V m_qx = A::fma(A::lit(-3), A::sub(h[1], h[3]), A::mul(two, jx));
  const V m_qy = A::fma(A::lit(-3), A::sub(h[2], h[4]), A::mul(two, jy));
  const V m_pxx = A::sub(A::sub(A::add(h[1], h[3]), A::add(h[2], h[4])),
                         A::mul(rho, A::mul(A::sub(ux, uy), A::add(ux, uy))));
  const V m_pxy = A::fma(A::mul(A::lit(-1), A::mul(rho, ux)), uy,
                         A::add(A::sub(h[5], h[6]), A::sub(h[7], h[8])));
  // relaxed amounts divided by the row norms
  using T = typename A::T;
  const V de = A::mul(A::splat((T)s.se * T(1.0 / 36.0)), m_e);
  const V deps = A::mul(A::splat((T)s.seps * T(1.0 / 36.0)), m_eps);
  const V dqx = A::mul(A::splat((T)s.sqx * T(1.0 / 12.0)), m_qx);
  const V dqy = A::mul(A::splat((T)s.sqy * T(1.0 / 12.0)), m_qy);
  const V dpxx = A::mul(A::splat((T)s.snxx * T(0.25)), m_pxx);
  const V dpxy = A::mul(A::splat((T)s.snxy * T(0.25)), m_pxy);
  // h* = h - M^T d (columns of M), with the sums the columns share
  const V e2 = A::fma(two, deps, de);            // de + 2 deps
  const V e5 = A::fma(two, de, deps);            // 2 de + deps
  h[0] = A::sub(h[0], A::mul(A::lit(4), A::sub(deps, de)));
  // axis directions: h1, h3 -= dpxx - e2 -+ 2 dqx; h2, h4 -= -(e2 + dpxx) -+ 2 dqy
  const V s13 = A::sub(dpxx, e2), s24 = A::mul(A::lit(-1), A::add(e2, dpxx));
  h[1] = A::sub(h[1], A::fma(A::lit(-2), dqx, s13));
  h[3] = A::sub(h[3], A::fma(two, dqx, s13));
  h[2] = A::sub(h[2], A::fma(A::lit(-2), dqy, s24));
  h[4] = A::sub(h[4], A::fma(two, dqy, s24));
  // diagonals: h5, h7 -= (e5 + dpxy) +- (dqx + dqy); h6, h8 -= (e5 - dpxy) +- (dqy - dqx)
  const V pp = A::add(e5, dpxy), pm = A::sub(e5, dpxy);
  const V a = A::add(dqx, dqy), b = A::sub(dqy, dqx);
  h[5] = A::sub(h[5], A::add(pp, a));
  h[7] = A::sub(h[7], A::sub(pp, a));
  h[6] = A::sub(h[6], A::add(pm, b));
  h[8] = A::sub(h[8], A::sub(pm, b));
  drho_out = drho; ux_out = ux; uy_out = uy;
}

// ---- Zou & He (Sec. 2.2) in shifted form ---------------------------------
// East side, prescribed density rho_out, zero tangential velocity (Eqs. 5-10).
// Known: 0, 1, 2, 4, 5, 8.  Unknown: 3, 6, 7.
template <typename R>
__device__ __forceinline__ void zouhe_east(R h[9], R rho_out) {
  // rho0 + 2 rho+ - 1 in shifted populations (the weights sum to exactly 1)
  const R s = (h[0] + h[2] + h[4]) + R(2) * (h[1] + h[5] + h[8]);
  const R u = (s + (R(1) - rho_out)) / rho_out;            // Eq. 7
  R heq[9];
  heq_sym(rho_out - R(1), u, R(0), heq);
  const R half_t = R(0.5) * ((h[4] - heq[4]) - (h[2] - heq[2]));
  h[3] = heq[3] + (h[1] - heq[1]);
  h[6] = heq[6] + (h[8] - heq[8]) + half_t;
  h[7] = heq[7] + (h[5] - heq[5]) - half_t;
}

// West side, prescribed velocity (u, v): the x-mirror of Eqs. 5-10.
// Known: 0, 2, 3, 4, 6, 7.  Unknown: 1, 5, 8.  rho (1 - u) = rho0 + 2 rho-.
template <typename R>
__device__ __forceinline__ void zouhe_west(R h[9], R u, R v) {
  const R s = (h[0] + h[2] + h[4]) + R(2) * (h[3] + h[6] + h[7]);
  const R drho = (s + u) / (R(1) - u);
  R heq[9];
  heq_sym(drho, u, v, heq);
  const R half_t = R(0.5) * ((h[4] - heq[4]) - (h[2] - heq[2]));
  h[1] = heq[1] + (h[3] - heq[3]);
  h[5] = heq[5] + (h[7] - heq[7]) + half_t;
  h[8] = heq[8] + (h[6] - heq[6]) - half_t;
}

// inlet velocity of step t: u_in, ramped linearly over the first ramp_steps
__device__ __forceinline__ double inlet_velocity(double u_in, int64_t ramp_steps, int64_t t) {
  if (ramp_steps <= 0 || t + 1 >= ramp_steps) return u_in;
  return u_in * ((double)(t + 1) / (double)ramp_steps);
}

// ---- SplitMix64 (Steele, Lea, Flood 2014), device copy --------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t key) {
  uint64_t z = key + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// inlet v(y, t) = amp (2 xi - 1), xi = top 53 bits of splitmix64(seed ^ (t 2^20 + y)) / 2^53
__device__ __forceinline__ double inlet_perturbation(uint64_t seed, int64_t t, int y, double amp) {
  const uint64_t z = splitmix64(seed ^ ((uint64_t)t * (1ull << 20) + (uint64_t)y));
  const double xi = (double)(z >> 11) * (1.0 / 9007199254740992.0);
  return amp * (2.0 * xi - 1.0);
}

}  // namespace lbm
