// In-place ("AA") stream-and-collide step on one population buffer (Bailey,
// Myre, Walsh, Lilja and Wilson, ICPP 2009).
//
// The AB step pulls every node's incoming populations from one buffer and
// writes the collided ones to another.  The AA step keeps one buffer whose
// slots alternate between two layouts:
//   after an even number of steps  slot opp(i) of x holds f*_i(x);
//   after an odd number            slot i of x + c_i holds f*_i(x).
// From an even count a node reads its incoming populations, f*_i(x - c_i) in
// slot opp(i) of x - c_i, collides, and writes f*_i(x) to slot i of x + c_i;
// from an odd count it reads slot i of x (which then holds f*_i(x - c_i)),
// collides, and writes f*_i(x) to slot opp(i) of x.  Either way every slot a
// node writes is read by that node alone in the same step, so the update is
// race-free in place: 72 B of traffic per node and step (FP32) as the AB step,
// with half its population memory.
//
// Full-way bounce-back (Eq. 11) needs no writes: a solid node would store the
// reversed arrivals into the slots they came from, which already hold them.
// The momentum exchange of a counted link between a fluid node x and the solid
// node s = x + c_i (Eqs. 13-14: the population arriving at s now plus the one
// s sends back now) is read from slot i of s and slot opp(i) of x in either
// parity; both are read before anything of this step can overwrite them, and
// the fluid node sums them (the fluid-side link masks come from the geometry
// preparation).  Zou & He inlet and outflow rebuild the unknown populations as
// in the AB step; the populations that leave the lattice through an open x
// side are kept in one ghost column on each side, so the state can always be
// exported exactly.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lattice.cuh"
#include "sim.cuh"

#include "step_kernels.cuh"

namespace lbm {
namespace {

template <typename S>
__device__ __forceinline__ typename Compute<S>::R ld(const S* p) {
  // plain (coherent) loads: the buffer is written during the launch
  return to_r<typename Compute<S>::R>(*p);
}

// the nine incoming populations of node (x, y): from an even step count
// f*_i(x - c_i) in slot opp(i) of x - c_i, from an odd one slot i of x
template <typename S, typename R>
__device__ __forceinline__ void load_node(const S* P, int plane, int pitch, int ny, int x, int xm,
                                          int xp, int y, bool gather, R h[9]) {
  const int ym = y == 0 ? ny - 1 : y - 1;
  const int yp = y == ny - 1 ? 0 : y + 1;
  const int rc = y * pitch, rm = ym * pitch, rp = yp * pitch;
  if (gather) {
    h[0] = ld(P + 0 * plane + rc + x);
    h[1] = ld(P + 3 * plane + rc + xm);
    h[2] = ld(P + 4 * plane + rm + x);
    h[3] = ld(P + 1 * plane + rc + xp);
    h[4] = ld(P + 2 * plane + rp + x);
    h[5] = ld(P + 7 * plane + rm + xm);
    h[6] = ld(P + 8 * plane + rm + xp);
    h[7] = ld(P + 5 * plane + rp + xp);
    h[8] = ld(P + 6 * plane + rp + xm);
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] = ld(P + i * plane + rc + x);
  }
}

template <typename S, int COLL, int MINB, bool PF>
__global__ void __launch_bounds__(128, MINB) aa_step_kernel(const StepParams p) {
  using R = typename Compute<S>::R;
  pdl_launch_dependents();
  pdl_wait();
  const int64_t t = step_index(p);
  // the force-reduction block of the previous step comes first
  if ((int)blockIdx.x < p.n_members) {
    if (p.reduce_prev && t >= 1) reduce_force(p, (int)blockIdx.x, t - 1);
    return;
  }
  const int b = (int)blockIdx.x - p.n_members;
  const int nblocks = (int)gridDim.x - p.n_members;
  const Member& m = p.m0;
  const Scalars<R> sc(m);
  S* __restrict__ P = static_cast<S*>(m.buf[0]);
  const int plane = m.plane, pitch = m.pitch, nx = m.nx, ny = m.ny;
  const bool gather = (t & 1) == 0;   // from an even count: neighbours' slots in and out
  double fx = 0.0, fy = 0.0;
  bool touched = false, bad = false;
  const int strips = m.strip_count;
  const int stride = p.persistent ? nblocks : strips;
  for (int s = b; s < strips; s += stride) {
    const int tx = s % m.tiles_x;
    const int y0 = (s / m.tiles_x) * p.rows;
    const int y1 = min(y0 + p.rows, ny);
    const int x = (tx << 7) + threadIdx.x;
    if (x >= nx) continue;
    const bool west = !m.x_periodic && x == 0;
    const bool east = !m.x_periodic && x == nx - 1;
    // neighbour columns: periodic wrap, else the ghost columns -1 and nx
    const int xm = m.x_periodic && x == 0 ? nx - 1 : x - 1;
    const int xp = m.x_periodic && x == nx - 1 ? 0 : x + 1;
    const uint32_t bit = 1u << (x & 31);
    const uint32_t* sb = m.solid_bits + (x >> 5);
    const uint32_t* nb = m.near_bits + (x >> 5);
    // PF: one row of look-ahead (a node reads only slots that it alone writes
    // in this step, so the next row's loads may run ahead of this row's stores)
    R h[9];
    if (PF) load_node<S, R>(P, plane, pitch, ny, x, xm, xp, y0, gather, h);
    for (int y = y0; y < y1; ++y) {
      const bool more = PF && y + 1 < y1;
      R hn[9];
      if (more) load_node<S, R>(P, plane, pitch, ny, x, xm, xp, y + 1, gather, hn);
      if (!PF) load_node<S, R>(P, plane, pitch, ny, x, xm, xp, y, gather, h);
      const bool solid = (__ldg(sb + y * m.words_per_row) & bit) != 0;
      if (!solid) {
        const int ym = y == 0 ? ny - 1 : y - 1;
        const int yp = y == ny - 1 ? 0 : y + 1;
        const int rc = y * pitch, rm = ym * pitch, rp = yp * pitch;
        if (__ldg(nb + y * m.words_per_row) & bit) {
          // counted links of this fluid node to solid nodes s = x + c_i
          const unsigned lk = __ldg(m.links + (int64_t)y * nx + x);
          R sx = R(0), sy = R(0);
#pragma unroll
          for (int i = 1; i < 9; ++i) {
            if ((lk >> (i - 1)) & 1u) {
              const int xs = cx(i) > 0 ? xp : (cx(i) < 0 ? xm : x);
              const int rs = cy(i) > 0 ? rp : (cy(i) < 0 ? rm : rc);
              const R v = ld(P + i * plane + rs + xs) + ld(P + opp(i) * plane + rc + x) +
                          R(2) * wgt<R>(i);
              sx += R(cx(i)) * v;
              sy += R(cy(i)) * v;
            }
          }
          fx += (double)sx;
          fy += (double)sy;
          touched = true;
        }
        if (west) {
          const R v = m.v_amp != 0.0 ? (R)inlet_perturbation(m.seed, t, y, m.v_amp) : R(0);
          const R u = m.ramp_steps > 0 ? (R)inlet_velocity(m.u_in, m.ramp_steps, t) : sc.u_in;
          zouhe_west<R>(h, u, v);
        } else if (east) {
          zouhe_east<R>(h, sc.rho_out);
        }
        R drho, ux, uy;
        if (COLL == 0 || (COLL == 2 && m.coll == LBM_BGK))
          collide_bgk<R>(h, sc.omega, drho, ux, uy);
        else
          collide_mrt<R>(h, mrt_of<R>(m), drho, ux, uy);
        bad |= nonfinite(drho);
        if (gather) {
          // f*_i(x) into slot i of x + c_i
          P[0 * plane + rc + x] = from_r<S>(h[0]);
          P[1 * plane + rc + xp] = from_r<S>(h[1]);
          P[2 * plane + rp + x] = from_r<S>(h[2]);
          P[3 * plane + rc + xm] = from_r<S>(h[3]);
          P[4 * plane + rm + x] = from_r<S>(h[4]);
          P[5 * plane + rp + xp] = from_r<S>(h[5]);
          P[6 * plane + rp + xm] = from_r<S>(h[6]);
          P[7 * plane + rm + xm] = from_r<S>(h[7]);
          P[8 * plane + rm + xp] = from_r<S>(h[8]);
        } else {
#pragma unroll
          for (int i = 0; i < 9; ++i) P[opp(i) * plane + rc + x] = from_r<S>(h[i]);
        }
      }   // fluid node
      if (more) {
#pragma unroll
        for (int i = 0; i < 9; ++i) h[i] = hn[i];
      }
    }
  }
  write_partial(p, t, b, fx, fy, touched, bad, p.m0.status);
}

// variants 0, 1, 2: 8 resident blocks per SM with a row of look-ahead, 8
// without, 10 without
template <typename S, int COLL>
void launch_aa_c(const StepParams& p, int variant, int blocks, cudaStream_t s) {
  const int g = blocks + p.n_members;
  if (variant == 1) launch_pdl(aa_step_kernel<S, COLL, 8, false>, g, 128, 0, s, p);
  else if (variant == 2) launch_pdl(aa_step_kernel<S, COLL, 10, false>, g, 128, 0, s, p);
  else launch_pdl(aa_step_kernel<S, COLL, 8, true>, g, 128, 0, s, p);
}

template <typename S>
void launch_aa_s(int coll, const StepParams& p, int variant, int blocks, cudaStream_t s) {
  if (coll == LBM_BGK) launch_aa_c<S, 0>(p, variant, blocks, s);
  else if (coll == LBM_MRT) launch_aa_c<S, 1>(p, variant, blocks, s);
  else launch_aa_c<S, 2>(p, variant, blocks, s);
}

template <typename S, int COLL>
int occ_aa_c(int variant) {
  int per_sm = 0;
  cudaError_t e;
  if (variant == 1)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, aa_step_kernel<S, COLL, 8, false>,
                                                      128, 0);
  else if (variant == 2)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, aa_step_kernel<S, COLL, 10, false>,
                                                      128, 0);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, aa_step_kernel<S, COLL, 8, true>,
                                                      128, 0);
  return e == cudaSuccess ? per_sm : 0;
}

template <typename S>
int occ_aa(int coll, int variant) {
  if (coll == LBM_BGK) return occ_aa_c<S, 0>(variant);
  if (coll == LBM_MRT) return occ_aa_c<S, 1>(variant);
  return occ_aa_c<S, 2>(variant);
}

}  // namespace

void launch_aa(int prec, int coll, const StepParams& p, int variant, int blocks, cudaStream_t s) {
  if (prec == LBM_FP64) launch_aa_s<double>(coll, p, variant, blocks, s);
  else if (prec == LBM_FP32) launch_aa_s<float>(coll, p, variant, blocks, s);
  else launch_aa_s<__half>(coll, p, variant, blocks, s);
}

int aa_max_blocks(int prec, int coll, int variant) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = prec == LBM_FP64 ? occ_aa<double>(coll, variant)
                   : prec == LBM_FP32 ? occ_aa<float>(coll, variant)
                                      : occ_aa<__half>(coll, variant);
  return sms > 0 && per_sm > 0 ? sms * per_sm : 0;
}

}  // namespace lbm
