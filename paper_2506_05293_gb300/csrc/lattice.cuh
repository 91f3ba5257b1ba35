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

// The same equilibrium evaluated pairwise: for a direction i and its opposite
// ibar, c.u changes sign, so h^eq_i,ibar = s_i +- a_i with
// s_i = w_i (drho - 3/2 rho u.u + 9/2 rho (c_i.u)^2) and a_i = 3 w_i rho c_i.u.
template <typename R>
__device__ __forceinline__ void heq_sym(R drho, R ux, R uy, R heq[9]) {
  const R rho = R(1) + drho;
  const R base = drho - R(1.5) * rho * (ux * ux + uy * uy);
  const R r45 = R(4.5) * rho, r3 = R(3) * rho;
  heq[0] = wgt<R>(0) * base;
  {
    const R s = wgt<R>(1) * (base + r45 * ux * ux), a = wgt<R>(1) * r3 * ux;
    heq[1] = s + a;
    heq[3] = s - a;
  }
  {
    const R s = wgt<R>(2) * (base + r45 * uy * uy), a = wgt<R>(2) * r3 * uy;
    heq[2] = s + a;
    heq[4] = s - a;
  }
  const R up = ux + uy;   // c5 = (1, 1); c7 = -c5
  const R um = uy - ux;   // c6 = (-1, 1); c8 = -c6
  {
    const R s = wgt<R>(5) * (base + r45 * up * up), a = wgt<R>(5) * r3 * up;
    heq[5] = s + a;
    heq[7] = s - a;
  }
  {
    const R s = wgt<R>(6) * (base + r45 * um * um), a = wgt<R>(6) * r3 * um;
    heq[6] = s + a;
    heq[8] = s - a;
  }
}

// correctly rounded reciprocal
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// rho - 1 and momentum of shifted populations (sum w_i = 1, sum w_i c_i = 0)
template <typename R>
__device__ __forceinline__ void moments_shifted(const R h[9], R& drho, R& jx, R& jy) {
  drho = ((h[0] + h[2]) + (h[4] + h[1])) + ((h[3] + h[5]) + (h[6] + h[7])) + h[8];
  jx = (h[1] - h[3]) + (h[5] - h[6]) + (h[8] - h[7]);
  jy = (h[2] - h[4]) + (h[5] + h[6]) - (h[7] + h[8]);
}

// ---- collision operators -------------------------------------------------
// BGK (Eq. 2): h* = h - omega (h - h^eq), omega = 1 / tau.
template <typename R>
__device__ __forceinline__ void collide_bgk(R h[9], R omega, R& drho_out, R& ux_out, R& uy_out) {
  R drho, jx, jy;
  moments_shifted(h, drho, jx, jy);
  const R inv_rho = recip(R(1) + drho);
  const R ux = jx * inv_rho, uy = jy * inv_rho;
  R heq[9];
  heq_sym(drho, ux, uy, heq);
#pragma unroll
  for (int i = 0; i < 9; ++i) h[i] = h[i] - omega * (h[i] - heq[i]);
  drho_out = drho; ux_out = ux; uy_out = uy;
}

// MRT with Lallemand & Luo's orthogonal basis (rho, e, eps, jx, qx, jy, qy,
// pxx, pxy).  Only the six non-conserved moments of the non-equilibrium part
// n = h - h^eq relax, each at its own rate: h* = h - M^-1 S M n, and
// M^-1 = M^T diag(1 / |row_k|^2) with |row|^2 = (9, 36, 36, 6, 12, 6, 12, 4, 4).
template <typename R>
struct MrtRates { R se, seps, sqx, sqy, snxx, snxy; };

template <typename R>
__device__ __forceinline__ void collide_mrt(R h[9], const MrtRates<R>& s, R& drho_out, R& ux_out,
                                            R& uy_out) {
  R drho, jx, jy;
  moments_shifted(h, drho, jx, jy);
  const R inv_rho = recip(R(1) + drho);
  const R ux = jx * inv_rho, uy = jy * inv_rho;
  R n[9];
  heq_sym(drho, ux, uy, n);
#pragma unroll
  for (int i = 0; i < 9; ++i) n[i] = h[i] - n[i];
  // moments of n (rows of M written out; integer coefficients)
  const R axis = (n[1] + n[2]) + (n[3] + n[4]);
  const R diag = (n[5] + n[6]) + (n[7] + n[8]);
  const R m_e = R(-4) * n[0] - axis + R(2) * diag;
  const R m_eps = R(4) * n[0] - R(2) * axis + diag;
  const R m_qx = R(-2) * (n[1] - n[3]) + (n[5] - n[6] - n[7] + n[8]);
  const R m_qy = R(-2) * (n[2] - n[4]) + (n[5] + n[6] - n[7] - n[8]);
  const R m_pxx = (n[1] + n[3]) - (n[2] + n[4]);
  const R m_pxy = (n[5] - n[6]) + (n[7] - n[8]);
  // relaxed amounts divided by the row norms
  const R de = s.se * m_e * (R(1) / R(36));
  const R deps = s.seps * m_eps * (R(1) / R(36));
  const R dqx = s.sqx * m_qx * (R(1) / R(12));
  const R dqy = s.sqy * m_qy * (R(1) / R(12));
  const R dpxx = s.snxx * m_pxx * R(0.25);
  const R dpxy = s.snxy * m_pxy * R(0.25);
  // h* = h - M^T d (columns of M)
  h[0] -= R(-4) * de + R(4) * deps;
  h[1] -= -de - R(2) * deps - R(2) * dqx + dpxx;
  h[2] -= -de - R(2) * deps - R(2) * dqy - dpxx;
  h[3] -= -de - R(2) * deps + R(2) * dqx + dpxx;
  h[4] -= -de - R(2) * deps + R(2) * dqy - dpxx;
  h[5] -= R(2) * de + deps + dqx + dqy + dpxy;
  h[6] -= R(2) * de + deps - dqx + dqy - dpxy;
  h[7] -= R(2) * de + deps - dqx - dqy + dpxy;
  h[8] -= R(2) * de + deps + dqx - dqy - dpxy;
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
