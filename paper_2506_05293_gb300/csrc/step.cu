// Fused stream-and-collide step of the D2Q9 lattice Boltzmann method and its
// helper kernels (geometry preparation, initialisation, export, mass).
//
// One launch advances every member lattice of a launch table by one time step
// (Sec. 2.1, Eq. 1, order of Fig. 1) in pull form: every node reads its nine
// incoming populations h_i(x - c_i) from its source buffer and writes its nine
// post-collision populations to the destination buffer, so each population is
// read once and written once per step (72 B per node in FP32).
//   - solid nodes (bit set in the solid mask): full-way bounce-back (Eq. 11)
//     stores the reversed incoming populations; counted links add their
//     momentum exchange (Eqs. 13-14) to an FP64 force accumulator;
//   - west column (open x): Zou & He velocity inlet, then collision;
//   - east column (open x): Zou & He pressure outflow (Eqs. 5-10) then
//     collision, or left to the outflow kernel (NN);
//   - all other fluid nodes: BGK (Eq. 2) or MRT collision.
// The lattice is cut into strips of 128 columns x `rows` rows.  A launch table
// lists the member lattices (one simulation, or a batch of simulations of
// different sizes and parameters advanced together); each block handles one
// strip (or, for a single member, strides over its strips).  Each block writes
// an FP64 partial of its member's force; one extra block per member in the
// next launch (or a finalise launch) sums them in a fixed order into the
// member's force ring, so results are bitwise reproducible run to run.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lattice.cuh"
#include "sim.cuh"

namespace lbm {

template <typename S>
__device__ __forceinline__ S ldg(const S* p) { return __ldg(p); }

template <typename R>
__device__ __forceinline__ void warp_sum2(R& a, R& b) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, off);
    b += __shfl_down_sync(0xffffffffu, b, off);
  }
}

// Pull-load the nine incoming populations of node (x, y): h_i = A_i(x - c_i).
// Offsets are 32-bit: the library keeps 9 * plane below 2^31 elements.
template <typename S, typename R>
__device__ __forceinline__ void pull_row(const S* __restrict__ A, int plane, int rc, int rm,
                                         int rp, int x, int xm, int xp, R h[9]) {
  h[0] = to_r<R>(ldg(A + rc + x));
  h[1] = to_r<R>(ldg(A + 1 * plane + rc + xm));
  h[2] = to_r<R>(ldg(A + 2 * plane + rm + x));
  h[3] = to_r<R>(ldg(A + 3 * plane + rc + xp));
  h[4] = to_r<R>(ldg(A + 4 * plane + rp + x));
  h[5] = to_r<R>(ldg(A + 5 * plane + rm + xm));
  h[6] = to_r<R>(ldg(A + 6 * plane + rm + xp));
  h[7] = to_r<R>(ldg(A + 7 * plane + rp + xp));
  h[8] = to_r<R>(ldg(A + 8 * plane + rp + xm));
}

template <typename R>
__device__ __forceinline__ bool nonfinite(R v) { return !(fabs(v) < R(1e30)); }

// A member's scalars in the compute precision (FP32 copies are made on the
// host: GB300's FP64 pipe is narrow).
template <typename R> struct Scalars;
template <> struct Scalars<float> {
  float omega, u_in, rho_out;
  MrtRates<float> mrt;
  __device__ explicit Scalars(const Member& m)
      : omega(m.omega_f), u_in(m.u_in_f), rho_out(m.rho_out_f),
        mrt{m.mrt_f[0], m.mrt_f[1], m.mrt_f[2], m.mrt_f[3]} {}
};
template <> struct Scalars<double> {
  double omega, u_in, rho_out;
  MrtRates<double> mrt;
  __device__ explicit Scalars(const Member& m)
      : omega(m.omega), u_in(m.u_in), rho_out(m.rho_out),
        mrt{m.mrt_se, m.mrt_seps, m.mrt_sq, m.mrt_snu} {}
};

// Programmatic dependent launch: a step kernel lets the next one be
// scheduled early (it then does its set-up while this one drains) and waits
// for the previous step's grid to complete before it touches populations.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ int64_t step_index(const StepParams& p) {
  return p.t_base ? *p.t_base + p.t_offset : p.t;
}

// Fixed-order sum of member k's block partials of step tt into its force ring
// (one block of 128 threads).
__device__ void reduce_force(const StepParams& p, int k, int64_t tt) {
  __shared__ double s_x[8], s_y[8];
  const Member& m = p.members[k];
  const double* part = p.partials + (size_t)(tt & 1) * 2 * p.partial_stride;
  double ax = 0.0, ay = 0.0;
  for (int b = m.part_first + threadIdx.x; b < m.part_first + m.part_count; b += blockDim.x) {
    ax += part[2 * b];
    ay += part[2 * b + 1];
  }
  warp_sum2(ax, ay);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { s_x[warp] = ax; s_y[warp] = ay; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bx = 0.0, by = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { bx += s_x[w]; by += s_y[w]; }
    const int64_t slot = tt % m.ring_cap;
    m.ring[2 * slot] = bx;
    m.ring[2 * slot + 1] = by;
  }
}

// Solid node: momentum exchange over counted links (FP64), then full-way
// bounce-back store.  Shared by both kernel families.
template <typename S, typename R>
__device__ __forceinline__ void solid_node(const S* __restrict__ A, S* __restrict__ B,
                                           const Member& m, int x, int y, int o, const R h[9],
                                           double& fx, double& fy, bool& touched) {
  const unsigned lk = __ldg(m.links + (int64_t)y * m.nx + x);
  if (lk) {
    touched = true;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      if ((lk >> (i - 1)) & 1u) {
        // f_i arriving now + f_ibar that bounce-back stored here last step
        const double v = (double)h[i] + (double)to_r<R>(ldg(A + opp(i) * m.plane + o)) +
                         2.0 * wgt<double>(i);
        fx += cx(i) * v;
        fy += cy(i) * v;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) B[i * m.plane + o] = from_r<S>(h[opp(i)]);
}

// Fluid node: open boundaries, collision, store.
template <typename S, typename R, int COLL>
__device__ __forceinline__ void fluid_node(S* __restrict__ B, const Member& m,
                                           const Scalars<R>& sc, int64_t t, bool west,
                                           bool east, int y, int o, R h[9], bool& bad) {
  if (west) {
    const R v = m.v_amp != 0.0 ? (R)inlet_perturbation(m.seed, t, y, m.v_amp) : R(0);
    const R u = m.ramp_steps > 0 ? (R)inlet_velocity(m.u_in, m.ramp_steps, t) : sc.u_in;
    zouhe_west<R>(h, u, v);
  } else if (east) {
    zouhe_east<R>(h, sc.rho_out);
  }
  R drho, ux, uy;
  // COLL 0: BGK, 1: MRT, 2: the member's own choice (mixed batches)
  if (COLL == 0 || (COLL == 2 && m.coll == LBM_BGK))
    collide_bgk<R>(h, sc.omega, drho, ux, uy);
  else
    collide_mrt<R>(h, sc.mrt, drho, ux, uy);
  bad |= nonfinite(drho);
#pragma unroll
  for (int i = 0; i < 9; ++i) B[i * m.plane + o] = from_r<S>(h[i]);
}

// Block partial of the force (FP64 shuffles only where a counted link was hit)
// and one block-wide vote on non-finite densities.
__device__ __forceinline__ void write_partial(const StepParams& p, int64_t t, double fx, double fy,
                                              bool touched, bool bad, int* status) {
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, DEV_NONFINITE);
  double* part = p.partials + (size_t)(t & 1) * 2 * p.partial_stride;
  if (!__syncthreads_or(touched)) {
    if (threadIdx.x == 0) {
      part[2 * blockIdx.x] = 0.0;
      part[2 * blockIdx.x + 1] = 0.0;
    }
    return;
  }
  __shared__ double s_fx[8], s_fy[8];
  warp_sum2(fx, fy);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { s_fx[warp] = fx; s_fy[warp] = fy; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bx = 0.0, by = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { bx += s_fx[w]; by += s_fy[w]; }
    part[2 * blockIdx.x] = bx;
    part[2 * blockIdx.x + 1] = by;
  }
}

// ---- register-pipelined kernel ---------------------------------------------
// Each thread walks its column down a strip and prefetches the next row's
// populations and solid-mask word while the current row collides.  With one
// member (p.persistent) blocks stride over its strips on a grid sized to the
// resident capacity; otherwise each block handles exactly one strip of the
// member given by the strip table.
template <typename S, int COLL>
__device__ __forceinline__ void reg_strip(const StepParams& p, const Member& m,
                                          const Scalars<typename Compute<S>::R>& sc, int64_t t,
                                          int s, double& fx, double& fy, bool& touched,
                                          bool& bad) {
  using R = typename Compute<S>::R;
  const S* __restrict__ A = static_cast<const S*>(m.buf[p.q]);
  S* __restrict__ B = static_cast<S*>(m.buf[1 - p.q]);
  const int plane = m.plane, pitch = m.pitch, nx = m.nx, ny = m.ny;
  const int tx = s % m.tiles_x;
  const int y0 = (s / m.tiles_x) * p.rows;
  const int y1 = min(y0 + p.rows, ny);
  const int x = (tx << 7) + threadIdx.x;
  if (x >= nx) return;
  const bool west = !m.x_periodic && x == 0;
  const bool east = !m.x_periodic && x == nx - 1;
  if (east && m.east_mode == EAST_EXTERNAL) return;
  const int xm = x == 0 ? nx - 1 : x - 1;
  const int xp = x == nx - 1 ? 0 : x + 1;
  const uint32_t* bits = m.solid_bits + (x >> 5);
  const uint32_t bit = 1u << (x & 31);

  R h[9];
  uint32_t word;
  {
    const int ym = y0 == 0 ? ny - 1 : y0 - 1;
    const int yp = y0 + 1 == ny ? 0 : y0 + 1;
    pull_row<S, R>(A, plane, y0 * pitch, ym * pitch, yp * pitch, x, xm, xp, h);
    word = __ldg(bits + y0 * m.words_per_row);
  }
  for (int y = y0; y < y1; ++y) {
    R hn[9];
    uint32_t word_n = 0;
    const bool more = y + 1 < y1;
    if (more) {
      const int y2 = y + 1;
      const int yp = y2 + 1 == ny ? 0 : y2 + 1;
      pull_row<S, R>(A, plane, y2 * pitch, y * pitch, yp * pitch, x, xm, xp, hn);
      word_n = __ldg(bits + y2 * m.words_per_row);
    }
    const int o = y * pitch + x;
    if (word & bit)
      solid_node<S, R>(A, B, m, x, y, o, h, fx, fy, touched);
    else
      fluid_node<S, R, COLL>(B, m, sc, t, west, east, y, o, h, bad);
    if (more) {
#pragma unroll
      for (int i = 0; i < 9; ++i) h[i] = hn[i];
      word = word_n;
    }
  }
}

template <typename S, int COLL, int MINB>
__global__ void __launch_bounds__(128, MINB) step_kernel(const StepParams p) {
  using R = typename Compute<S>::R;
  pdl_launch_dependents();
  pdl_wait();
  const int nblocks = gridDim.x - p.n_members;
  const int64_t t = step_index(p);
  if ((int)blockIdx.x >= nblocks) {
    if (p.reduce_prev && t >= 1) reduce_force(p, (int)blockIdx.x - nblocks, t - 1);
    return;
  }
  double fx = 0.0, fy = 0.0;
  bool touched = false, bad = false;
  if (p.n_members == 1) {
    // the member lives in the parameter bank: no registers held for its fields
    const Scalars<R> sc(p.m0);
    const int strips = p.m0.strip_count;
    const int stride = p.persistent ? nblocks : strips;
    for (int s = blockIdx.x; s < strips; s += stride)
      reg_strip<S, COLL>(p, p.m0, sc, t, s, fx, fy, touched, bad);
    write_partial(p, t, fx, fy, touched, bad, p.m0.status);
  } else {
    const Member& m = p.members[p.strip_member[blockIdx.x]];
    const Scalars<R> sc(m);
    reg_strip<S, COLL>(p, m, sc, t, (int)blockIdx.x - m.strip_first, fx, fy, touched, bad);
    write_partial(p, t, fx, fy, touched, bad, m.status);
  }
}

__global__ void finalize_force_kernel(const StepParams p, int64_t tt) {
  reduce_force(p, blockIdx.x, tt);
}

__global__ void set_t_kernel(int64_t* t_base, int64_t value) { *t_base = value; }

void launch_finalize_force(const StepParams& p, int64_t tt, cudaStream_t s) {
  finalize_force_kernel<<<p.n_members, 128, 0, s>>>(p, tt);
}

void launch_set_t(int64_t* t_base, int64_t value, cudaStream_t s) {
  set_t_kernel<<<1, 1, 0, s>>>(t_base, value);
}

// ---- bulk-copy staged kernel -------------------------------------------------
// One block = one strip.  Thread 0 stages, for each output row, the nine
// source row segments (rows y - c_iy, columns shifted by -c_ix) plus the row's
// solid-mask words into a ring of NS shared-memory slots with cp.async.bulk
// copies that complete on one mbarrier per slot; all threads collide from
// shared memory and store coalesced rows.  Each staged segment starts A
// elements (16 bytes) before the tile, so every copy is 16-byte aligned and
// the x shifts become fixed offsets.  Waits are bounded: a wait that gives up
// latches DEV_TIMEOUT and the block drains its copies before it exits.

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// try_wait with a suspend-time hint: the thread sleeps in hardware until the
// phase completes or the hint (ns) elapses, instead of spinning
constexpr uint32_t kSuspendHintNs = 1000000;   // 1 ms per attempt

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendHintNs)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

constexpr uint32_t kWaitLimit = 2000;   // attempts (x the 1 ms hint) before a wait gives up

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (uint32_t k = 0; k < kWaitLimit; ++k)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

template <typename S>
struct BulkLayout {
  static constexpr int A = 16 / (int)sizeof(S);      // 16 bytes in elements
  static constexpr int SEG = 128 + A;                // staged elements per source row
  static constexpr int SEG_BYTES = SEG * (int)sizeof(S);
  static constexpr int STAGE_BYTES = 9 * SEG_BYTES + 16;   // + 4 solid-mask words
  static constexpr uint32_t TX_BYTES = (uint32_t)STAGE_BYTES;
};

size_t step_bulk_smem(int prec, int stages) {
  const int sb = prec == LBM_FP64 ? BulkLayout<double>::STAGE_BYTES
               : prec == LBM_FP32 ? BulkLayout<float>::STAGE_BYTES
                                  : BulkLayout<__half>::STAGE_BYTES;
  return (size_t)stages * sb + (size_t)stages * 16 + 16;   // ring + full/empty barriers
}

// One block streams the rows of its strips (local strips lb, lb + gk, ... of
// member m) through an NS-slot ring with warp specialisation: warp 4 is the
// producer -- its lane 0 waits until a slot is released ("empty" barrier,
// one arrival per consumer warp), then stages the next row into it with
// cp.async.bulk completing on the slot's "full" barrier -- and warps 0-3 are
// consumers, each waiting on "full", colliding its 32 columns and releasing
// the slot.  No block-wide barrier per row: warps run ahead independently.
constexpr int kConsumerWarps = 4;
constexpr int kBulkThreads = 32 * (kConsumerWarps + 1);

template <typename S, int COLL, int NS>
__device__ __forceinline__ void bulk_run(const StepParams& p, const Member& m, int lb, int gk,
                                         unsigned char* smem) {
  using R = typename Compute<S>::R;
  using Lay = BulkLayout<S>;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NS * Lay::STAGE_BYTES);
  uint64_t* empty = full + NS;
  __shared__ int s_abort;
  const S* __restrict__ A = static_cast<const S*>(m.buf[p.q]);
  S* __restrict__ B = static_cast<S*>(m.buf[1 - p.q]);
  const int plane = m.plane, pitch = m.pitch;
  const int nx = m.nx, ny = m.ny, tiles_x = m.tiles_x, rows = p.rows;
  const int strips = m.strip_count;
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
  // set-up done: wait for the previous step to complete before touching the
  // populations (it may still be reading the buffer this step writes)
  pdl_wait();
  const int64_t t = step_index(p);

  // strip geometry
  struct Strip {
    int y0, x0, lead, nrows;
  };
  auto strip_at = [&](int ls) {
    Strip st;
    st.y0 = (ls / tiles_x) * rows;
    st.x0 = (ls % tiles_x) << 7;
    st.lead = st.x0 == 0 ? 0 : Lay::A;
    st.nrows = min(rows, ny - st.y0);
    return st;
  };

  double fx = 0.0, fy = 0.0;
  bool touched = false, bad = false;

  if (warp == kConsumerWarps) {
    // ---------------- producer ----------------
    if ((threadIdx.x & 31) == 0) {
      int ps = lb, pr = 0, k = 0;
      Strip pst = strip_at(lb);
      while (ps < strips) {
        const int slot = k % NS;
        if (k >= NS && !mbar_wait_bounded(&empty[slot], (uint32_t)(((k / NS) - 1) & 1))) {
          atomicOr(m.status, DEV_TIMEOUT);
          s_abort = 1;
          break;
        }
        if (s_abort) break;
        const int y = pst.y0 + pr;
        unsigned char* st = smem + slot * Lay::STAGE_BYTES;
        mbar_expect_tx(&full[slot], Lay::TX_BYTES);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          int sy = y - cy(i);
          sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
          const int sx = cx(i) == 1 ? pst.x0 - pst.lead : pst.x0;
          bulk_copy_g2s(st + i * Lay::SEG_BYTES, A + i * plane + sy * pitch + sx,
                        (uint32_t)Lay::SEG_BYTES, &full[slot]);
        }
        bulk_copy_g2s(st + 9 * Lay::SEG_BYTES,
                      m.solid_bits + y * m.words_per_row + (pst.x0 >> 5), 16u, &full[slot]);
        ++k;
        if (++pr == pst.nrows) {
          pr = 0;
          ps += gk;
          if (ps < strips) pst = strip_at(ps);
        }
      }
      // no copy may land after the block exits: wait (bounded) for the last
      // item staged into each slot
      for (int kk = k > NS ? k - NS : 0; kk < k; ++kk)
        mbar_wait_bounded(&full[kk % NS], (uint32_t)((kk / NS) & 1));
    }
  } else {
    // ---------------- consumers ----------------
    const int lx = threadIdx.x;     // column within the 128-wide tile
    const Scalars<R> sc(m);
    int cs = lb, cr = 0, j = 0;
    Strip cst = strip_at(lb);
    int x = cst.x0 + lx;
    bool west = !m.x_periodic && x == 0;
    bool east = !m.x_periodic && x == nx - 1;
    bool skip = x >= nx || (east && m.east_mode == EAST_EXTERNAL);
    while (cs < strips) {
      const int slot = j % NS;
      // warp-uniform outcome, so the warp never diverges around __syncwarp
      const bool ready = __all_sync(
          0xffffffffu, !s_abort && mbar_wait_bounded(&full[slot], (uint32_t)((j / NS) & 1)));
      if (!ready) {
        atomicOr(m.status, DEV_TIMEOUT);
        s_abort = 1;
        break;
      }
      const int y = cst.y0 + cr;
      const unsigned char* st = smem + slot * Lay::STAGE_BYTES;
      if (!skip) {
        const S* seg = reinterpret_cast<const S*>(st);
        R h[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          const int idx = cx(i) == 1 ? lx - 1 + cst.lead : (cx(i) == 0 ? lx : lx + 1);
          h[i] = to_r<R>(seg[i * Lay::SEG + (idx < 0 ? 0 : idx)]);
        }
        if (x == 0 || x == nx - 1) {
          // periodic wrap of the x +- 1 neighbours at the lattice edges
          const int ym = y == 0 ? ny - 1 : y - 1;
          const int yp = y == ny - 1 ? 0 : y + 1;
          if (x == 0) {
            h[1] = to_r<R>(A[1 * plane + y * pitch + nx - 1]);
            h[5] = to_r<R>(A[5 * plane + ym * pitch + nx - 1]);
            h[8] = to_r<R>(A[8 * plane + yp * pitch + nx - 1]);
          }
          if (x == nx - 1) {
            h[3] = to_r<R>(A[3 * plane + y * pitch]);
            h[6] = to_r<R>(A[6 * plane + ym * pitch]);
            h[7] = to_r<R>(A[7 * plane + yp * pitch]);
          }
        }
        const uint32_t word =
            reinterpret_cast<const uint32_t*>(st + 9 * Lay::SEG_BYTES)[lx >> 5];
        const int o = y * pitch + x;
        if ((word >> (lx & 31)) & 1u)
          solid_node<S, R>(A, B, m, x, y, o, h, fx, fy, touched);
        else
          fluid_node<S, R, COLL>(B, m, sc, t, west, east, y, o, h, bad);
      }
      __syncwarp();
      if ((threadIdx.x & 31) == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[slot]))
                     : "memory");
      ++j;
      if (++cr == cst.nrows) {
        cr = 0;
        cs += gk;
        if (cs < strips) {
          cst = strip_at(cs);
          x = cst.x0 + lx;
          west = !m.x_periodic && x == 0;
          east = !m.x_periodic && x == nx - 1;
          skip = x >= nx || (east && m.east_mode == EAST_EXTERNAL);
        }
      }
    }
  }
  write_partial(p, t, fx, fy, touched, bad, m.status);
}

template <typename S, int COLL, int NS, int MINB>
__global__ void __launch_bounds__(kBulkThreads, MINB) step_bulk_kernel(const StepParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  pdl_launch_dependents();
  const int nblocks = gridDim.x - p.n_members;
  if ((int)blockIdx.x >= nblocks) {
    pdl_wait();
    const int64_t t = step_index(p);
    if (p.reduce_prev && t >= 1) reduce_force(p, (int)blockIdx.x - nblocks, t - 1);
    return;
  }
  if (p.n_members == 1) {
    // blocks part_count apart share the strips: part_count = strips gives one
    // strip per block, fewer blocks make them stream several strips each
    bulk_run<S, COLL, NS>(p, p.m0, (int)blockIdx.x, p.m0.part_count, smem);
  } else {
    // stage this block's member record in shared memory once (coalesced),
    // instead of every thread chasing its fields in global memory
    __shared__ __align__(16) Member s_member;
    constexpr int kWords = (int)(sizeof(Member) / sizeof(uint64_t));
    static_assert(sizeof(Member) % sizeof(uint64_t) == 0, "Member must be 8-byte sized");
    if (threadIdx.x < 32) {
      const uint64_t* src =
          reinterpret_cast<const uint64_t*>(p.members + p.strip_member[blockIdx.x]);
      uint64_t* dst = reinterpret_cast<uint64_t*>(&s_member);
      for (int w = threadIdx.x; w < kWords; w += 32) dst[w] = src[w];
    }
    __syncthreads();
    bulk_run<S, COLL, NS>(p, s_member, (int)blockIdx.x - s_member.part_first,
                          s_member.part_count, smem);
  }
}

// ---- variants and launch ------------------------------------------------------
int step_strips(int nx, int ny, int rows) {
  return ((nx + 127) / 128) * ((ny + rows - 1) / rows);
}

// Variants 0-2: the register-pipelined kernel with __launch_bounds__ minimum
// resident blocks of 128 threads per SM of 6, 8, 10.  Variant 3: the
// warp-specialised staged kernel (4-slot ring), one block per strip.
// Variant 4: the same on a resident-sized grid, each block streaming several
// strips through its ring.
constexpr int kVariants = 5;
constexpr int kBulkSlots = 4;

bool step_variant_is_bulk(int variant) { return variant >= 3; }
bool step_variant_streams(int variant) { return variant >= 4; }

int step_variants() { return kVariants; }

template <typename S>
static constexpr int prec_of() {
  return sizeof(S) == 8 ? LBM_FP64 : (sizeof(S) == 4 ? LBM_FP32 : LBM_FP16DEV);
}

template <typename S, int COLL, int MINB>
static cudaError_t occ_bulk(int* per_sm) {
  const size_t smem = step_bulk_smem(prec_of<S>(), kBulkSlots);
  auto k = step_bulk_kernel<S, COLL, kBulkSlots, MINB>;
  const cudaError_t e =
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, kBulkThreads, smem);
}

template <typename S, int COLL>
static cudaError_t occ(int variant, int* per_sm) {
  switch (variant) {
    case 0: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, step_kernel<S, COLL, 6>, 128, 0);
    case 1: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, step_kernel<S, COLL, 8>, 128, 0);
    case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, step_kernel<S, COLL, 10>, 128, 0);
    default: return occ_bulk<S, COLL, 6>(per_sm);
  }
}

int step_max_blocks(int prec, int coll, int variant) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  auto by_coll = [&](auto tag) {
    using S = decltype(tag);
    return coll == 0 ? occ<S, 0>(variant, &per_sm)
                     : (coll == 1 ? occ<S, 1>(variant, &per_sm) : occ<S, 2>(variant, &per_sm));
  };
  if (prec == LBM_FP64) e = by_coll(double{});
  else if (prec == LBM_FP32) e = by_coll(float{});
  else e = by_coll(__half{});
  if (e != cudaSuccess || sms <= 0 || per_sm <= 0) return 0;
  return sms * per_sm;
}

// Launch with programmatic stream serialisation (dependent launch).
template <typename Kernel>
static void launch_pdl(Kernel kernel, int grid, int threads, size_t smem, cudaStream_t s,
                       const StepParams& p) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, p);
}

template <typename S, int COLL, int MINB>
static void launch_bulk(const StepParams& p, int blocks, cudaStream_t s) {
  // the dynamic shared memory attribute is set by the occupancy query that
  // every group runs at creation (occ_bulk)
  const size_t smem = step_bulk_smem(prec_of<S>(), kBulkSlots);
  launch_pdl(step_bulk_kernel<S, COLL, kBulkSlots, MINB>, blocks + p.n_members, kBulkThreads,
             smem, s, p);
}

template <typename S, int COLL>
static void launch_v(const StepParams& p, int variant, int blocks, cudaStream_t s) {
  const int g = blocks + p.n_members;
  switch (variant) {
    case 0: launch_pdl(step_kernel<S, COLL, 6>, g, 128, 0, s, p); break;
    case 1: launch_pdl(step_kernel<S, COLL, 8>, g, 128, 0, s, p); break;
    case 2: launch_pdl(step_kernel<S, COLL, 10>, g, 128, 0, s, p); break;
    default: launch_bulk<S, COLL, 6>(p, blocks, s); break;
  }
}

template <typename S>
static void launch_c(int coll, const StepParams& p, int variant, int blocks, cudaStream_t s) {
  if (coll == LBM_BGK) launch_v<S, 0>(p, variant, blocks, s);
  else if (coll == LBM_MRT) launch_v<S, 1>(p, variant, blocks, s);
  else launch_v<S, 2>(p, variant, blocks, s);
}

void launch_step(int prec, int coll, const StepParams& p, int variant, int blocks, cudaStream_t s) {
  if (prec == LBM_FP64) launch_c<double>(coll, p, variant, blocks, s);
  else if (prec == LBM_FP32) launch_c<float>(coll, p, variant, blocks, s);
  else launch_c<__half>(coll, p, variant, blocks, s);
}

// ---- geometry preparation --------------------------------------------------
// One thread per 32-cell word of a row: packs the solid bits and, for every
// counted solid node, the mask of links to fluid neighbours s - c_i.
__global__ void geometry_prep_kernel(const uint8_t* __restrict__ kind, int nx, int ny,
                                     int x_periodic, uint32_t* bits, int wpr,
                                     uint8_t* links) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (w >= wpr || y >= ny) return;
  uint32_t word = 0;
  for (int b = 0; b < 32; ++b) {
    const int x = w * 32 + b;
    if (x >= nx) break;
    const uint8_t k = kind[(int64_t)y * nx + x];
    if (k != LBM_CELL_FLUID) word |= 1u << b;
    uint8_t lk = 0;
    if (k == LBM_CELL_SOLID) {
      for (int i = 1; i < 9; ++i) {
        int sx = x - cx(i);
        int sy = y - cy(i);
        sy = (sy + ny) % ny;
        if (sx < 0 || sx >= nx) {
          if (!x_periodic) continue;
          sx = (sx + nx) % nx;
        }
        if (kind[(int64_t)sy * nx + sx] == LBM_CELL_FLUID) lk |= (uint8_t)(1u << (i - 1));
      }
    }
    links[(int64_t)y * nx + x] = lk;
  }
  bits[(int64_t)y * wpr + w] = word;
}

void launch_geometry_prep(const uint8_t* kind, int nx, int ny, int x_periodic, uint32_t* bits,
                          int words_per_row, uint8_t* links, cudaStream_t s) {
  dim3 grid((words_per_row + 127) / 128, ny);
  geometry_prep_kernel<<<grid, 128, 0, s>>>(kind, nx, ny, x_periodic, bits, words_per_row, links);
}

// ---- initialisation, import and export --------------------------------------
template <typename S>
__global__ void init_eq_kernel(S* dst, int nx, int ny, int64_t pitch, int64_t plane,
                               const double* rho, const double* ux, const double* uy) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= nx) return;
  const int64_t c = (int64_t)y * nx + x;
  const double r = rho ? rho[c] : 1.0;
  const double u = ux ? ux[c] : 0.0;
  const double v = uy ? uy[c] : 0.0;
  double heq[9];
  heq_all<double>(r - 1.0, u, v, heq);
  for (int i = 0; i < 9; ++i) dst[i * plane + (int64_t)y * pitch + x] = from_r<S>(heq[i]);
}

void launch_init_equilibrium(int prec, void* dst, int nx, int ny, int64_t pitch, int64_t plane,
                             const double* rho, const double* ux, const double* uy,
                             cudaStream_t s) {
  dim3 grid((nx + 127) / 128, ny);
  if (prec == LBM_FP64)
    init_eq_kernel<double><<<grid, 128, 0, s>>>((double*)dst, nx, ny, pitch, plane, rho, ux, uy);
  else if (prec == LBM_FP32)
    init_eq_kernel<float><<<grid, 128, 0, s>>>((float*)dst, nx, ny, pitch, plane, rho, ux, uy);
  else
    init_eq_kernel<__half><<<grid, 128, 0, s>>>((__half*)dst, nx, ny, pitch, plane, rho, ux, uy);
}

// f_i = h_i + w_i into a dense double[9][ny][nx]; moments into rho/ux/uy.
template <typename S>
__global__ void export_kernel(const S* src, int nx, int ny, int64_t pitch, int64_t plane,
                              double* f_out, double* rho, double* ux, double* uy) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= nx) return;
  const int64_t c = (int64_t)y * nx + x;
  const int64_t n = (int64_t)nx * ny;
  double f[9];
  for (int i = 0; i < 9; ++i) {
    f[i] = (double)to_r<double>(src[i * plane + (int64_t)y * pitch + x]) + wgt<double>(i);
    if (f_out) f_out[i * n + c] = f[i];
  }
  double r = 0.0, jx = 0.0, jy = 0.0;
  for (int i = 0; i < 9; ++i) {
    r += f[i];
    jx += cx(i) * f[i];
    jy += cy(i) * f[i];
  }
  if (rho) rho[c] = r;
  if (ux) ux[c] = jx / r;
  if (uy) uy[c] = jy / r;
}

void launch_export(int prec, const void* src, int nx, int ny, int64_t pitch, int64_t plane,
                   double* f_out, double* rho, double* ux, double* uy, cudaStream_t s) {
  dim3 grid((nx + 127) / 128, ny);
  if (prec == LBM_FP64)
    export_kernel<double><<<grid, 128, 0, s>>>((const double*)src, nx, ny, pitch, plane, f_out,
                                               rho, ux, uy);
  else if (prec == LBM_FP32)
    export_kernel<float><<<grid, 128, 0, s>>>((const float*)src, nx, ny, pitch, plane, f_out, rho,
                                              ux, uy);
  else
    export_kernel<__half><<<grid, 128, 0, s>>>((const __half*)src, nx, ny, pitch, plane, f_out,
                                               rho, ux, uy);
}

template <typename S>
__global__ void import_kernel(S* dst, int nx, int ny, int64_t pitch, int64_t plane,
                              const double* f_in) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= nx) return;
  const int64_t c = (int64_t)y * nx + x;
  const int64_t n = (int64_t)nx * ny;
  for (int i = 0; i < 9; ++i)
    dst[i * plane + (int64_t)y * pitch + x] = from_r<S>(f_in[i * n + c] - wgt<double>(i));
}

void launch_import(int prec, void* dst, int nx, int ny, int64_t pitch, int64_t plane,
                   const double* f_in, cudaStream_t s) {
  dim3 grid((nx + 127) / 128, ny);
  if (prec == LBM_FP64)
    import_kernel<double><<<grid, 128, 0, s>>>((double*)dst, nx, ny, pitch, plane, f_in);
  else if (prec == LBM_FP32)
    import_kernel<float><<<grid, 128, 0, s>>>((float*)dst, nx, ny, pitch, plane, f_in);
  else
    import_kernel<__half><<<grid, 128, 0, s>>>((__half*)dst, nx, ny, pitch, plane, f_in);
}

// ---- total mass: per-row partial sums, then one block sums the rows --------
template <typename S>
__global__ void mass_rows_kernel(const S* src, int nx, int ny, int64_t pitch, int64_t plane,
                                 double* partials) {
  const int y = blockIdx.x;
  double acc = 0.0;
  for (int x = threadIdx.x; x < nx; x += blockDim.x) {
    double cell = 1.0;   // sum of the weights
    for (int i = 0; i < 9; ++i) cell += (double)to_r<double>(src[i * plane + (int64_t)y * pitch + x]);
    acc += cell;
  }
  __shared__ double sh[32];
  double dummy = 0.0;
  warp_sum2(acc, dummy);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    partials[y] = s;
  }
}

__global__ void sum_partials_kernel(const double* partials, int n, double* out) {
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) acc += partials[k];
  __shared__ double sh[32];
  double dummy = 0.0;
  warp_sum2(acc, dummy);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    *out = s;
  }
}

void launch_mass(int prec, const void* src, int nx, int ny, int64_t pitch, int64_t plane,
                 double* partials, int n_partials, double* out, cudaStream_t s) {
  (void)n_partials;
  if (prec == LBM_FP64)
    mass_rows_kernel<double><<<ny, 256, 0, s>>>((const double*)src, nx, ny, pitch, plane, partials);
  else if (prec == LBM_FP32)
    mass_rows_kernel<float><<<ny, 256, 0, s>>>((const float*)src, nx, ny, pitch, plane, partials);
  else
    mass_rows_kernel<__half><<<ny, 256, 0, s>>>((const __half*)src, nx, ny, pitch, plane, partials);
  sum_partials_kernel<<<1, 1024, 0, s>>>(partials, ny, out);
}

}  // namespace lbm
