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

// ---- staged in-place kernel (variant 3) ---------------------------------------
// One block per strip, warp-specialised like the two-buffer staged kernel: a
// producer lane copies, per output row, the nine source row segments the
// row's nodes read -- from an even step count slot opp(i) of row y - c_iy,
// from an odd one slot i of row y -- into a ring of shared-memory slots with
// cp.async.bulk, and four consumer warps collide from it and store in place.
// A segment spans columns x0 - 1 .. x0 + 128 (+ padding): the buffer starts
// one element before column 0 (the ghost column -1), so that column x0 - 1
// lies on a 16-byte boundary for every tile.  Reads staged ahead of this
// step's stores are safe: every slot a node writes is read by that node alone
// within the step (the in-place invariant), before it writes.
template <typename S>
struct AaLayout {
  static constexpr int A = 16 / (int)sizeof(S);
  static constexpr int SEG = 128 + 2 * A;          // columns x0 - 1 .. x0 + 128, padded
  static constexpr int SEG_BYTES = SEG * (int)sizeof(S);
  static constexpr int STAGE_BYTES = 9 * SEG_BYTES + 16;   // + the row's solid-mask words
};
constexpr int kAaSlots = 4;

template <typename S, int COLL>
__global__ void __launch_bounds__(kBulkThreads, 6) aa_bulk_kernel(const StepParams p) {
  using R = typename Compute<S>::R;
  using Lay = AaLayout<S>;
  constexpr int NS = kAaSlots;
  extern __shared__ __align__(128) unsigned char smem[];
  pdl_launch_dependents();
  // the force-reduction block of the previous step comes first
  if ((int)blockIdx.x < p.n_members) {
    pdl_wait();
    const int64_t t = step_index(p);
    if (p.reduce_prev && t >= 1) reduce_force(p, (int)blockIdx.x, t - 1);
    return;
  }
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NS * Lay::STAGE_BYTES);
  uint64_t* empty = full + NS;
  __shared__ int s_abort;
  const Member& m = p.m0;
  S* P = static_cast<S*>(m.buf[0]);
  const int plane = m.plane, pitch = m.pitch, nx = m.nx, ny = m.ny;
  const int b = (int)blockIdx.x - p.n_members;
  const int sg = p.strip_order ? p.strip_order[b] : b;   // strips holding solids first
  const int y0 = (sg / m.tiles_x) * p.rows;
  const int x0 = (sg % m.tiles_x) << 7;
  const int nrows = min(p.rows, ny - y0);
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int k = 0; k < NS; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // the previous step must be complete before anything of this one is read
  pdl_wait();
  const int64_t t = step_index(p);
  const bool gather = (t & 1) == 0;   // from an even count: neighbours' slots in and out
  double fx = 0.0, fy = 0.0;
  bool touched = false, bad = false;

  if (warp == kConsumerWarps) {
    // ---------------- producer ----------------
    if ((threadIdx.x & 31) == 0) {
      int k = 0;
      for (int r = 0; r < nrows; ++r, ++k) {
        const int slot = k % NS;
        if (k >= NS && !mbar_wait_bounded(&empty[slot], (uint32_t)(((k / NS) - 1) & 1))) {
          atomicOr(m.status, DEV_TIMEOUT);
          s_abort = 1;
          break;
        }
        if (s_abort) break;
        const int y = y0 + r;
        unsigned char* st = smem + slot * Lay::STAGE_BYTES;
        mbar_expect_tx(&full[slot], (uint32_t)Lay::STAGE_BYTES);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          int sy = gather ? y - cy(i) : y;
          sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
          const int slot_i = gather ? opp(i) : i;
          bulk_copy_g2s(st + i * Lay::SEG_BYTES, P + slot_i * plane + sy * pitch + x0 - 1,
                        (uint32_t)Lay::SEG_BYTES, &full[slot]);
        }
        bulk_copy_g2s(st + 9 * Lay::SEG_BYTES, m.solid_bits + y * m.words_per_row + (x0 >> 5),
                      16u, &full[slot]);
      }
      // no copy may land after the block exits
      for (int kk = k > NS ? k - NS : 0; kk < k; ++kk)
        mbar_wait_bounded(&full[kk % NS], (uint32_t)((kk / NS) & 1));
    }
  } else {
    // ---------------- consumers ----------------
    const int lx = threadIdx.x;     // column within the 128-wide tile
    const int lane = threadIdx.x & 31;
    const int x = x0 + lx;
    const Scalars<R> sc(m);
    const bool skip = x >= nx;
    const bool west = !m.x_periodic && x == 0;
    const bool east = !m.x_periodic && x == nx - 1;
    // neighbour columns: periodic wrap, else the ghost columns -1 and nx
    const int xm = m.x_periodic && x == 0 ? nx - 1 : x - 1;
    const int xp = m.x_periodic && x == nx - 1 ? 0 : x + 1;
    // with a periodic x the edge columns' x -+ 1 neighbours are the opposite
    // edge, not the staged ghost columns: those nodes read the buffer itself
    const bool wrap = m.x_periodic && (x == 0 || x == nx - 1);
    const uint32_t bit = 1u << (x & 31);
    const uint32_t* nb = m.near_bits + (x >> 5);
    for (int r = 0; r < nrows; ++r) {
      const int slot = r % NS;
      // warp-uniform outcome, so the warp never diverges around __syncwarp
      const bool ready = __all_sync(
          0xffffffffu, !s_abort && mbar_wait_bounded(&full[slot], (uint32_t)((r / NS) & 1)));
      if (!ready) {
        atomicOr(m.status, DEV_TIMEOUT);
        s_abort = 1;
        break;
      }
      const int y = y0 + r;
      const unsigned char* st = smem + slot * Lay::STAGE_BYTES;
      const uint32_t word = reinterpret_cast<const uint32_t*>(st + 9 * Lay::SEG_BYTES)[lx >> 5];
      // a solid node needs no writes: its reversed arrivals already sit in
      // the slots they came from
      if (!skip && !((word >> (lx & 31)) & 1u)) {
        const int ym = y == 0 ? ny - 1 : y - 1;
        const int yp = y == ny - 1 ? 0 : y + 1;
        const int rc = y * pitch, rm = ym * pitch, rp = yp * pitch;
        R h[9];
        if (wrap) {
          load_node<S, R>(P, plane, pitch, ny, x, xm, xp, y, gather, h);
        } else {
          const S* seg = reinterpret_cast<const S*>(st);
#pragma unroll
          for (int i = 0; i < 9; ++i)
            h[i] = to_r<R>(seg[i * Lay::SEG + lx + 1 - (gather ? cx(i) : 0)]);
        }
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
      }
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[slot]))
                     : "memory");
    }
  }
  const int fslot = p.strip_force ? p.strip_force[sg] : sg;
  write_partial(p, t, fslot, fx, fy, touched, bad, m.status);
}

size_t aa_bulk_smem(int prec) {
  const int sb = prec == LBM_FP64 ? AaLayout<double>::STAGE_BYTES
               : prec == LBM_FP32 ? AaLayout<float>::STAGE_BYTES
                                  : AaLayout<__half>::STAGE_BYTES;
  return (size_t)kAaSlots * sb + (size_t)kAaSlots * 16;   // ring + full/empty barriers
}

// variants 0, 1, 2: 8 resident blocks per SM with a row of look-ahead, 8
// without, 10 without; variant 3: the staged kernel, one block per strip
template <typename S, int COLL>
void launch_aa_c(const StepParams& p, int variant, int blocks, cudaStream_t s) {
  const int g = blocks + p.n_members;
  if (variant == 3)
    launch_pdl(aa_bulk_kernel<S, COLL>, g, kBulkThreads, aa_bulk_smem(prec_of<S>()), s, p);
  else if (variant == 1) launch_pdl(aa_step_kernel<S, COLL, 8, false>, g, 128, 0, s, p);
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
  if (variant == 3)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, aa_bulk_kernel<S, COLL>,
                                                      kBulkThreads, aa_bulk_smem(prec_of<S>()));
  else if (variant == 1)
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
