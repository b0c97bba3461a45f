// Pipelined persistent Dhop: neighbour rows streamed into a ring of shared-memory slots by bulk
// asynchronous copies (TMA), several copies in flight while the CTA computes.
//
// Why: the direct kernel gathers each neighbour spinor with ordinary loads; six of the eight
// hops miss L1 and wait ~1000 cycles on L2, and the registers of a thread cannot hold the next
// hop's loads while it computes the current one, so the SMs idle on latency (ncu: long-
// scoreboard stalls, 14 warps per SM). Here the loads are issued by one thread as bulk copies of
// whole x-rows, ahead of use, and cost no registers.
//
// Work unit (tile): R consecutive x-rows of output sites, R dividing Ly, so that all rows of a
// tile share (z, t) and the checkerboard index range of the tile is contiguous. One thread per
// (site, slice pair). A tile is consumed in stages; each stage is one ring slot of R rows:
//   X   the tile's own rows of the input field (both x hops: x-neighbours never leave the row),
//   YH  the two y-halo rows y0 - 1 and y0 + R (R >= 2; the interior y-neighbours are in X),
//       or Y+ and Y- as two stages of one row each (R = 1),
//   Z+, Z-, T+, T-  the tile's rows shifted by one in z or t (with wrap-around),
//   AUX the tile's rows of the epilogue input field (only when there is a pre-epilogue).
// Rows read per output row: 5 + 2/R for R >= 2 (the direct kernel gathers 8 neighbour sites
// per output site). The links of a tile (8 per site) are fetched one tile ahead with per-thread
// 16-byte asynchronous copies into a double buffer.
//
// Status: correct (parity-tested like the direct kernel) but measured slower on GB300 at
// 16^4 x 16 (FP32 55-61 us against 34 us for the direct kernel): shared memory limits the CTA
// to 8-12 resident warps, too few to hide the shared-memory and FMA latencies of the hops, and
// the bulk copies deliver about 5 TB/s in aggregate. It is therefore opt-in (GRID_DWF_PIPE=1).
//
// Ring protocol: stage g of this CTA (g counts across its tiles) lives in slot g mod NS and
// completes on that slot's mbarrier, phase (g / NS) mod 2. One thread issues every copy. A
// slot is refilled with stage g + NS once every thread has finished with stage g (a CTA
// barrier, then a proxy fence); X is held until the y hops of YH are done. Every wait has an
// iteration limit: on timeout the CTA sets bit 0 of *status, waits (bounded) for the copies it
// issued, and returns.
#pragma once

#include "dhop_tma.cuh"

namespace gdwf {

enum PipeStage { ST_X = 0, ST_YH, ST_YP, ST_YM, ST_ZP, ST_ZM, ST_TP, ST_TM, ST_AUX };

__host__ __device__ inline int pipe_stage_kind(int R, int st) {
  // R >= 2: X, YH, Z+, Z-, T+, T-, AUX;  R = 1: X, Y+, Y-, Z+, Z-, T+, T-, AUX
  if (R >= 2) return st < 2 ? st : st + 2;
  return st == 0 ? ST_X : st + 1;
}

// Shared-memory plan of one CTA (byte offsets), shared by the host launcher and the kernel.
struct PipePlan {
  int R;                     // x-rows per tile
  int slots;                 // ring slots
  int spt;                   // stages per tile
  int tiles;                 // tiles in the half lattice
  unsigned site_bytes;       // padded Ls * 24 * sizeof(storage)
  unsigned row_bytes;        // Lx/2 site blocks
  unsigned slot_bytes;       // R rows
  unsigned link_tile_bytes;  // 8 links per site of a tile
  unsigned off_links;        // two link buffers
  unsigned off_scratch;      // Mooee^-1 epilogue scratch (a slot is reused when it is large enough)
  unsigned scratch_bytes;    // 0: the epilogue reuses the last stage's slot
  unsigned off_bars;         // one mbarrier per slot
  unsigned bytes;            // total
};

__host__ __device__ inline PipePlan pipe_plan(const Geom& g, int R, int slots, int real_bytes, int LB, bool aux,
                                              bool post) {
  PipePlan p;
  p.R = R;
  p.slots = slots;
  p.spt = (R >= 2 ? 6 : 7) + (aux ? 1 : 0);
  p.tiles = g.N4h / (R * g.Lxh);
  p.site_bytes = (unsigned)ls_padded(g.Ls) * 24u * (unsigned)real_bytes;
  p.row_bytes = (unsigned)g.Lxh * p.site_bytes;
  p.slot_bytes = (unsigned)R * p.row_bytes;
  p.link_tile_bytes = (unsigned)(R * g.Lxh) * 8u * (unsigned)LB;
  p.off_links = (unsigned)slots * p.slot_bytes;
  p.off_scratch = p.off_links + 2u * p.link_tile_bytes;
  const unsigned need = post ? (unsigned)(R * g.Lxh) * (unsigned)g.Ls * 24u * 4u : 0u;
  p.scratch_bytes = need > p.slot_bytes ? need : 0u;
  p.off_bars = (p.off_scratch + p.scratch_bytes + 15u) / 16u * 16u;
  p.bytes = p.off_bars + ((unsigned)slots * 8u + 15u) / 16u * 16u;
  return p;
}

__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// (y, z, t) of x-row rho.
__device__ __forceinline__ void pipe_row_coords(const Geom& g, int rho, int& y, int& z, int& t) {
  const uint32_t r1 = fdiv((uint32_t)rho, g.div_ly);
  y = rho - (int)r1 * g.L[1];
  const uint32_t r2 = fdiv(r1, g.div_lz);
  z = (int)r1 - (int)r2 * g.L[2];
  t = (int)r2;
}

// Issue the copies of stage gs into its slot (one thread); nothing past the last stage.
template <int P>
__device__ __forceinline__ void pipe_issue(const DhopArgs& a, const PipePlan& pl, unsigned char* smem, uint64_t* bars,
                                           long gs, long nst) {
  if (gs >= nst) return;
  const Geom& g = a.g;
  const int n = (int)(gs / pl.spt);
  const int st = (int)(gs - (long)n * pl.spt);
  const int tile = blockIdx.x + n * gridDim.x;
  const int R = pl.R;
  const int rho0 = tile * R;
  int y0, z, t;
  pipe_row_coords(g, rho0, y0, z, t);
  const int slot = (int)(gs % pl.slots);
  unsigned char* dst = smem + (size_t)slot * pl.slot_bytes;
  uint64_t* bar = bars + slot;
  const char* in = static_cast<const char*>(a.in);
  const int Ly = g.L[1], Lz = g.L[2], Lt = g.L[3];
  const int rowy = rho0 - y0;  // row of y = 0 at this (z, t)
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  switch (pipe_stage_kind(R, st)) {
    case ST_X:
      mbar_arrive_expect_tx(bar, pl.slot_bytes);
      bulk_g2s(dst, in + (size_t)rho0 * pl.row_bytes, pl.slot_bytes, bar);
      break;
    case ST_YH: {
      const int rm = rowy + (y0 == 0 ? Ly - 1 : y0 - 1);
      const int rp = rowy + (y0 + R == Ly ? 0 : y0 + R);
      mbar_arrive_expect_tx(bar, 2u * pl.row_bytes);
      bulk_g2s(dst, in + (size_t)rm * pl.row_bytes, pl.row_bytes, bar);
      bulk_g2s(dst + pl.row_bytes, in + (size_t)rp * pl.row_bytes, pl.row_bytes, bar);
      break;
    }
    case ST_YP:
    case ST_YM: {
      const bool fwd = pipe_stage_kind(R, st) == ST_YP;
      const int rr = rowy + (fwd ? (y0 == Ly - 1 ? 0 : y0 + 1) : (y0 == 0 ? Ly - 1 : y0 - 1));
      mbar_arrive_expect_tx(bar, pl.row_bytes);
      bulk_g2s(dst, in + (size_t)rr * pl.row_bytes, pl.row_bytes, bar);
      break;
    }
    case ST_ZP:
    case ST_ZM:
    case ST_TP:
    case ST_TM: {
      const int kind = pipe_stage_kind(R, st);
      int shift;
      if (kind == ST_ZP) shift = (z == Lz - 1 ? -(Lz - 1) : 1) * Ly;
      else if (kind == ST_ZM) shift = (z == 0 ? (Lz - 1) : -1) * Ly;
      else if (kind == ST_TP) shift = (t == Lt - 1 ? -(Lt - 1) : 1) * Ly * Lz;
      else shift = (t == 0 ? (Lt - 1) : -1) * Ly * Lz;
      mbar_arrive_expect_tx(bar, pl.slot_bytes);
      bulk_g2s(dst, in + (size_t)(rho0 + shift) * pl.row_bytes, pl.slot_bytes, bar);
      break;
    }
    default: {  // ST_AUX
      const char* aux = static_cast<const char*>(a.aux);
      mbar_arrive_expect_tx(bar, pl.slot_bytes);
      bulk_g2s(dst, aux + (size_t)rho0 * pl.row_bytes, pl.slot_bytes, bar);
      break;
    }
  }
}

// Bounded wait of every thread for stage gs; false if the limit was reached.
__device__ __forceinline__ bool pipe_wait(uint64_t* bars, const PipePlan& pl, long gs) {
  uint64_t* bar = bars + (int)(gs % pl.slots);
  const unsigned phase = (unsigned)((gs / pl.slots) & 1);
  unsigned long long it = 0;
  while (!mbar_try_wait(bar, phase)) {
    if (++it > TMA_WAIT_LIMIT) return false;
  }
  return true;
}

// Per-thread 16-byte asynchronous copies of the links of one tile: thread q of a site takes the
// hops q, q + Lsh, ... (hop h = 2 mu + backward).
template <int P, bool C12>
__device__ __forceinline__ void pipe_fetch_links(const DhopArgs& a, const PipePlan& pl, unsigned char* lbuf, int tile,
                                                 int sl, int r, int k, int q, int Lsh) {
  using T = typename Store<P>::T;
  constexpr int LB = link_bytes(sizeof(T), C12);
  const Geom& g = a.g;
  const int rho = tile * pl.R + r;
  const int site = rho * g.Lxh + k;
  int c[4];
  pipe_row_coords(g, rho, c[1], c[2], c[3]);
  c[0] = 2 * k + ((a.out_parity + c[1] + c[2] + c[3]) & 1);
  const char* Uo = static_cast<const char*>(a.Uout);
  const char* Ui = static_cast<const char*>(a.Uin);
  for (int h = q; h < 8; h += Lsh) {
    const int mu = h >> 1;
    const char* src;
    if ((h & 1) == 0) {
      src = Uo + ((size_t)site * 4 + mu) * LB;
    } else {
      int ph;
      src = Ui + ((size_t)cb_neighbour(g, site, c, mu, false, ph) * 4 + mu) * LB;
    }
    unsigned char* dst = lbuf + ((size_t)sl * 8 + h) * LB;
#pragma unroll
    for (int b = 0; b < LB / 16; ++b) cp_async16(dst + 16 * b, src + 16 * b);
  }
}

// One hop from a staged block: (1 + S gamma_mu) U psi with U or U^+ (backward), scaled.
template <int P, bool C12, int S, bool BACK, int LSH>
__device__ __forceinline__ void pipe_hop(int mu, const unsigned char* blk, const unsigned char* lnk, int q, float scale,
                                         float2* acc) {
  float u[18];
  load_link_smem<P, C12>(reinterpret_cast<const char*>(lnk), u);
  float2 psi[24], h[12], uh[12];
  load_pair<P, LSH, false>(reinterpret_cast<const char*>(blk), q, LSH, psi);
  project2<S>(mu, psi, h);
  su3_mul2<BACK>(u, h, uh);
  accumulate2<S>(mu, uh, scale, acc);
}

template <int P, bool DAG, bool C12, int LSC>
__device__ __forceinline__ void dhop_pipe_body(const DhopArgs& a) {
  using T = typename Store<P>::T;
  constexpr int LB = link_bytes(sizeof(T), C12);
  constexpr int SF = DAG ? +1 : -1;
  constexpr int SB = -SF;
  constexpr int Ls = LSC;
  constexpr int Lsh = ls_half(LSC);
  const Geom& g = a.g;
  const PipePlan pl =
      pipe_plan(g, a.pipe_rows, a.pipe_slots, (int)sizeof(T), LB, a.pre != PRE_NONE, a.post != POST_NONE);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + pl.off_bars);
  unsigned char* lbuf0 = smem_raw + pl.off_links;

  const int tid = threadIdx.x;
  const int R = pl.R;
  const int sl = tid / Lsh;  // site within the tile
  const int q = tid - sl * Lsh;
  const int r = sl / g.Lxh;  // row within the tile
  const int k = sl - r * g.Lxh;
  const int ntiles = (pl.tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const long nst = (long)ntiles * pl.spt;
  const float alpha = (float)a.alpha;
  const size_t gsite_bytes = pl.site_bytes;

  if (tid == 0) {
    for (int s = 0; s < pl.slots; ++s) mbar_init(bars + s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  long issued = 0;  // meaningful in thread 0 only
  if (tid == 0) {
    for (; issued < pl.slots && issued < nst; ++issued) pipe_issue<P>(a, pl, smem_raw, bars, issued, nst);
  }
  if (ntiles > 0) pipe_fetch_links<P, C12>(a, pl, lbuf0, blockIdx.x, sl, r, k, q, Lsh);
  cp_async_commit();

  bool failed = false;
  long gs = 0;
  for (int n = 0; n < ntiles && !failed; ++n) {
    const int tile = blockIdx.x + n * gridDim.x;
    const int rho = tile * R + r;
    const int site = rho * g.Lxh + k;
    int c[4];
    pipe_row_coords(g, rho, c[1], c[2], c[3]);
    c[0] = 2 * k + ((a.out_parity + c[1] + c[2] + c[3]) & 1);
    unsigned char* lbuf = lbuf0 + (size_t)(n & 1) * pl.link_tile_bytes;
    cp_async_wait_all();
    __syncthreads();
    if (n + 1 < ntiles) {
      pipe_fetch_links<P, C12>(a, pl, lbuf0 + (size_t)((n + 1) & 1) * pl.link_tile_bytes, tile + gridDim.x, sl, r, k,
                               q, Lsh);
      cp_async_commit();
    }
    const unsigned char* lnk = lbuf + (size_t)sl * 8 * LB;

    float2 acc[24];
#pragma unroll
    for (int i = 0; i < 24; ++i) acc[i] = make_float2(0.f, 0.f);

    for (int st = 0; st < pl.spt; ++st, ++gs) {
      const bool ok = pipe_wait(bars, pl, gs);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      const unsigned char* slot = smem_raw + (size_t)(gs % pl.slots) * pl.slot_bytes;
      const int kind = pipe_stage_kind(R, st);
      if (kind == ST_X) {
        int xn = c[0] + 1, ph = 1;
        if (xn == g.L[0]) {
          xn = 0;
          ph = g.bc[0];
        }
        pipe_hop<P, C12, SF, false, Lsh>(0, slot + (size_t)(r * g.Lxh + (xn >> 1)) * gsite_bytes, lnk, q,
                                         ph < 0 ? -alpha : alpha, acc);
        xn = c[0] - 1;
        ph = 1;
        if (xn < 0) {
          xn = g.L[0] - 1;
          ph = g.bc[0];
        }
        pipe_hop<P, C12, SB, true, Lsh>(0, slot + (size_t)(r * g.Lxh + (xn >> 1)) * gsite_bytes, lnk + LB, q,
                                        ph < 0 ? -alpha : alpha, acc);
      } else if (kind == ST_YH) {
        const unsigned char* xs = smem_raw + (size_t)((gs - 1) % pl.slots) * pl.slot_bytes;
        const unsigned char* bp = r < R - 1 ? xs + (size_t)((r + 1) * g.Lxh + k) * gsite_bytes
                                            : slot + (size_t)(g.Lxh + k) * gsite_bytes;
        const unsigned char* bm =
            r > 0 ? xs + (size_t)((r - 1) * g.Lxh + k) * gsite_bytes : slot + (size_t)k * gsite_bytes;
        const float sp = (c[1] == g.L[1] - 1 && g.bc[1] < 0) ? -alpha : alpha;
        const float sm = (c[1] == 0 && g.bc[1] < 0) ? -alpha : alpha;
        pipe_hop<P, C12, SF, false, Lsh>(1, bp, lnk + 2 * LB, q, sp, acc);
        pipe_hop<P, C12, SB, true, Lsh>(1, bm, lnk + 3 * LB, q, sm, acc);
      } else if (kind != ST_AUX) {
        int mu, fwd;
        switch (kind) {
          case ST_YP: mu = 1; fwd = 1; break;
          case ST_YM: mu = 1; fwd = 0; break;
          case ST_ZP: mu = 2; fwd = 1; break;
          case ST_ZM: mu = 2; fwd = 0; break;
          case ST_TP: mu = 3; fwd = 1; break;
          default: mu = 3; fwd = 0; break;
        }
        const unsigned char* b = slot + (size_t)((R >= 2 ? r : 0) * g.Lxh + k) * gsite_bytes;
        const bool edge = fwd ? c[mu] == g.L[mu] - 1 : c[mu] == 0;
        const float sc = (edge && g.bc[mu] < 0) ? -alpha : alpha;
        if (fwd)
          pipe_hop<P, C12, SF, false, Lsh>(mu, b, lnk + (2 * mu) * LB, q, sc, acc);
        else
          pipe_hop<P, C12, SB, true, Lsh>(mu, b, lnk + (2 * mu + 1) * LB, q, sc, acc);
      } else {  // pre-epilogue from the staged aux rows
        const unsigned char* ab = slot + (size_t)sl * gsite_bytes;
        const float2 B = f2((float)a.beta);
        if (a.pre == PRE_AUX) {
          float2 o[24];
          load_pair<P, Lsh, false>(reinterpret_cast<const char*>(ab), q, Lsh, o);
#pragma unroll
          for (int i = 0; i < 24; ++i) acc[i] = ffma2(B, o[i], acc[i]);
        } else {
          float o0[24], o1[24];
          const char* abc = reinterpret_cast<const char*>(ab);
          if (a.pre == PRE_MOOEE) {
            mooee_slice<P, false, false>(abc, 2 * q, Ls, Lsh, a.d5, a.mass, o0);
            mooee_slice<P, false, false>(abc, 2 * q + 1, Ls, Lsh, a.d5, a.mass, o1);
          } else {
            mooee_slice<P, true, false>(abc, 2 * q, Ls, Lsh, a.d5, a.mass, o0);
            mooee_slice<P, true, false>(abc, 2 * q + 1, Ls, Lsh, a.d5, a.mass, o1);
          }
#pragma unroll
          for (int i = 0; i < 24; ++i) acc[i] = ffma2(B, make_float2(o0[i], o1[i]), acc[i]);
        }
      }

      if (st == pl.spt - 1) {
        // ------------------------------------------------ epilogue of the tile
        const bool pad_lane = (Ls & 1) && q == Lsh - 1;
        char* outb = static_cast<char*>(a.out) + (size_t)site * gsite_bytes;
        if (a.post == POST_NONE) {
          if (pad_lane) {
#pragma unroll
            for (int i = 0; i < 24; ++i) acc[i].y = 0.f;
          }
          store_pair<P, Lsh>(outb, q, Lsh, acc);
        } else {
          // the last stage's slot is free once every thread has read it
          __syncthreads();
          float* sm = reinterpret_cast<float*>(pl.scratch_bytes ? smem_raw + pl.off_scratch
                                                                : smem_raw + (size_t)(gs % pl.slots) * pl.slot_bytes);
          float* d0 = sm + ((size_t)sl * Ls + 2 * q) * 24;
#pragma unroll
          for (int i = 0; i < 24; ++i) d0[i] = acc[i].x;
          if (!pad_lane) {
#pragma unroll
            for (int i = 0; i < 24; ++i) d0[24 + i] = acc[i].y;
          }
          __syncthreads();
          const int S = R * g.Lxh;
          for (int task = tid; task < S * 24; task += blockDim.x) {
            const int ts = task / 24;
            const int ri = task - ts * 24;
            const bool upper = ri < 12;
            const bool forward_form = (a.post == POST_INV) ? upper : !upper;
            mooee_inv_line<float>(sm + (size_t)ts * Ls * 24 + ri, Ls, forward_form, (float)a.mass, (float)a.inv_d5,
                                  (float)a.inv_den);
          }
          __syncthreads();
          const float* s0 = sm + ((size_t)sl * Ls + 2 * q) * 24;
#pragma unroll
          for (int i = 0; i < 24; ++i) acc[i] = make_float2(s0[i], pad_lane ? 0.f : s0[24 + i]);
          store_pair<P, Lsh>(outb, q, Lsh, acc);
        }
      }

      __syncthreads();  // every thread is done with this stage's slot (and, after YH, with X's)
      if (tid == 0) {
        if (R >= 2 && kind == ST_X) {
          // X stays resident until the y hops of the next stage
        } else if (R >= 2 && kind == ST_YH) {
          pipe_issue<P>(a, pl, smem_raw, bars, gs - 1 + pl.slots, nst);
          pipe_issue<P>(a, pl, smem_raw, bars, gs + pl.slots, nst);
          issued = gs + pl.slots + 1;
        } else {
          pipe_issue<P>(a, pl, smem_raw, bars, gs + pl.slots, nst);
          issued = gs + pl.slots + 1;
        }
        if (issued > nst) issued = nst;
      }
    }
  }
  cp_async_wait_all();
  if (failed && tid == 0) {
    if (a.status) atomicOr(a.status, 1);
    // let every copy this CTA issued land before its shared memory is released
    for (long w = gs; w < issued; ++w) {
      uint64_t* bar = bars + (int)(w % pl.slots);
      const unsigned phase = (unsigned)((w / pl.slots) & 1);
      unsigned long long it = 0;
      while (!mbar_try_wait(bar, phase) && ++it < TMA_WAIT_LIMIT) {
      }
    }
  }
}

template <int P, bool DAG, bool C12, int LSC>
__global__ void __launch_bounds__(128) dhop_pipe_kernel(const __grid_constant__ DhopArgs a) {
  dhop_pipe_body<P, DAG, C12, LSC>(a);
}

// Host: choose rows per tile and ring slots for a geometry, or 0 when the pipelined kernel does
// not apply (then the direct kernel runs). Threads per CTA = R * Lx/2 * Lsh, at most 256; R
// divides Ly; the plan must fit the opt-in shared memory of one CTA.
inline int pipe_choose_rows(const Geom& g, int real_bytes, int LB, bool aux, bool post, int max_smem, int& slots) {
  const int Lsh = ls_half(g.Ls);
  int best = 0;
  for (int R = 1; R <= 8; ++R) {
    if (g.L[1] % R != 0) continue;
    const int threads = R * g.Lxh * Lsh;
    if (threads > 128) break;
    const PipePlan p = pipe_plan(g, R, 3, real_bytes, LB, aux, post);
    if ((int)p.bytes > max_smem) break;
    best = R;
  }
  slots = 3;
  return best;
}

}  // namespace gdwf
