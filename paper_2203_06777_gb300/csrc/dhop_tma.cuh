// Dhop with the neighbour data staged by the Tensor Memory Accelerator (bulk asynchronous
// copies into shared memory), for lattices whose x-rows split into segments of whole sites.
//
// Why: in the direct kernel every thread loads its eight neighbour spinors through L1, which
// hits only for the x hops; the other six come from L2 with ~1000-cycle latency on the two-die
// part, and registers cannot hold enough loads in flight to cover it. Here one CTA owns a
// segment of `seg` consecutive checkerboard sites of one x-row (all slices, one thread per
// (site, slice pair), packed two-wide arithmetic as in the direct kernel). Because the cb index runs x-fastest, each neighbour row-segment is one
// contiguous run of site blocks in memory, so the CTA needs only a handful of bulk copies:
//   x hops:            seg + 2 site blocks of the same row (x - 1 ... x + seg, wrapping),
//   y, z, t hops:      seg site blocks of each of the six neighbour rows,
//   links:             the segment's own links (forward hops), and the input-parity links of the
//                      x-range and of the rows at -y, -z, -t (backward hops).
// One thread issues all copies against one mbarrier (expect_tx = total bytes); every thread
// waits on it with an iteration limit (on timeout the CTA records an error in *status, waits
// once more, bounded, for its copies and returns), then computes the eight hops from shared
// memory exactly as the direct kernel does, with the same epilogues (the Mooee^-1 epilogue
// reuses the staged buffers once all hops are done).
#pragma once

#include "dhop_kernel.cuh"

namespace gdwf {

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16) completing on bar.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

constexpr unsigned long long TMA_WAIT_LIMIT = 1ull << 24;  // try_wait rounds before giving up

// Shared-memory plan of one CTA (byte offsets), shared by the host launcher and the kernel.
struct TmaPlan {
  int seg;               // sites per CTA
  unsigned site_bytes;   // padded Ls * 24 * sizeof(storage)
  unsigned lrow_bytes;   // 4 links of one site
  unsigned off_x;        // seg + 2 site blocks
  unsigned off_rows;     // 6 * seg site blocks, rows in the order y+, y-, z+, z-, t+, t-
  unsigned off_lfwd;     // seg link rows (output parity)
  unsigned off_lbx;      // seg + 2 link rows (input parity, x range)
  unsigned off_lbr;      // 3 * seg link rows (input parity, rows -y, -z, -t)
  unsigned bytes;        // total, including the mbarrier at the end
};

__host__ __device__ inline TmaPlan tma_plan(int seg, int Ls, int real_bytes, int link_b) {
  TmaPlan p;
  p.seg = seg;
  p.site_bytes = (unsigned)ls_padded(Ls) * 24u * (unsigned)real_bytes;
  p.lrow_bytes = 4u * (unsigned)link_b;
  p.off_x = 0;
  p.off_rows = p.off_x + (unsigned)(seg + 2) * p.site_bytes;
  p.off_lfwd = p.off_rows + 6u * (unsigned)seg * p.site_bytes;
  p.off_lbx = p.off_lfwd + (unsigned)seg * p.lrow_bytes;
  p.off_lbr = p.off_lbx + (unsigned)(seg + 2) * p.lrow_bytes;
  const unsigned end = p.off_lbr + 3u * (unsigned)seg * p.lrow_bytes;
  p.bytes = (end + 15u) / 16u * 16u + 16u;  // mbarrier in the last 16 bytes
  return p;
}

// Copy `count` consecutive site-sized records of a row starting at row position `first`
// (wrapping modulo the row length lxh) into dst; at most two bulk copies. Returns bytes issued.
__device__ __forceinline__ unsigned copy_row_run(char* dst, const char* row_base, int first, int count, int lxh,
                                                 unsigned rec_bytes, uint64_t* bar) {
  unsigned issued = 0;
  int pos = ((first % lxh) + lxh) % lxh;
  int left = count;
  while (left > 0) {
    const int run = min(left, lxh - pos);
    bulk_g2s(dst, row_base + (size_t)pos * rec_bytes, (unsigned)run * rec_bytes, bar);
    issued += (unsigned)run * rec_bytes;
    dst += (size_t)run * rec_bytes;
    left -= run;
    pos = 0;
  }
  return issued;
}

template <int P, bool DAG, bool C12, int LSC>
__device__ __forceinline__ void dhop_tma_body(const DhopArgs& a) {
  using T = typename Store<P>::T;
  constexpr int LB = link_bytes(sizeof(T), C12);
  constexpr int SF = DAG ? +1 : -1;
  constexpr int Ls = LSC;
  constexpr int Lsh = ls_half(LSC);
  const Geom& g = a.g;
  const int seg = a.seg;
  const TmaPlan pl = tma_plan(seg, Ls, (int)sizeof(T), LB);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + pl.bytes - 16);

  const int tid = threadIdx.x;
  const int sl = tid / Lsh;  // site within the segment
  const int q = tid - sl * Lsh;
  const int segs_per_row = g.Lxh / seg;
  const int row = blockIdx.x / segs_per_row;
  const int a0 = (blockIdx.x - row * segs_per_row) * seg;  // first xh of the segment
  const int row_base = row * g.Lxh;                       // cb index of xh = 0 in this row
  const int site = row_base + a0 + sl;

  // row coordinates (y, z, t) and the neighbour rows
  const uint32_t r1 = fdiv((uint32_t)row, g.div_ly);
  const int y = row - (int)r1 * g.L[1];
  const uint32_t r2 = fdiv(r1, g.div_lz);
  const int z = (int)r1 - (int)r2 * g.L[2];
  const int t = (int)r2;
  const int L1 = g.L[1], L2 = g.L[2], L3 = g.L[3];
  const int rows_pm[6] = {
      row + (y == L1 - 1 ? -(L1 - 1) : 1),            // y+
      row + (y == 0 ? (L1 - 1) : -1),                 // y-
      row + (z == L2 - 1 ? -(L2 - 1) : 1) * L1,       // z+
      row + (z == 0 ? (L2 - 1) : -1) * L1,            // z-
      row + (t == L3 - 1 ? -(L3 - 1) : 1) * L1 * L2,  // t+
      row + (t == 0 ? (L3 - 1) : -1) * L1 * L2,       // t-
  };

  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  __syncthreads();
  const char* in = static_cast<const char*>(a.in);
  const char* Uo = static_cast<const char*>(a.Uout);
  const char* Ui = static_cast<const char*>(a.Uin);
  if (tid == 0) {
    const unsigned sb = pl.site_bytes, lr = pl.lrow_bytes;
    const unsigned total =
        (unsigned)(seg + 2) * sb + 6u * seg * sb + (unsigned)seg * lr + (unsigned)(seg + 2) * lr + 3u * seg * lr;
    mbar_arrive_expect_tx(bar, total);
    // spinors: x range of this row, then the segment's xh range in the six neighbour rows
    copy_row_run(reinterpret_cast<char*>(smem_raw + pl.off_x), in + (size_t)row_base * sb, a0 - 1, seg + 2, g.Lxh,
                 sb, bar);
#pragma unroll
    for (int k = 0; k < 6; ++k)
      bulk_g2s(smem_raw + pl.off_rows + (unsigned)k * seg * sb, in + ((size_t)rows_pm[k] * g.Lxh + a0) * sb,
               (unsigned)seg * sb, bar);
    // links: forward (output parity, this segment), backward x range and rows -y, -z, -t (input parity)
    bulk_g2s(smem_raw + pl.off_lfwd, Uo + (size_t)(row_base + a0) * lr, (unsigned)seg * lr, bar);
    copy_row_run(reinterpret_cast<char*>(smem_raw + pl.off_lbx), Ui + (size_t)row_base * lr, a0 - 1, seg + 2, g.Lxh,
                 lr, bar);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      bulk_g2s(smem_raw + pl.off_lbr + (unsigned)k * seg * lr, Ui + ((size_t)rows_pm[2 * k + 1] * g.Lxh + a0) * lr,
               (unsigned)seg * lr, bar);
  }

  // every thread: coordinates and boundary phases of its output site
  int c[4];
  c[1] = y;
  c[2] = z;
  c[3] = t;
  c[0] = 2 * (a0 + sl) + ((a.out_parity + y + z + t) & 1);
  const float alpha = (float)a.alpha;

  bool ok = true;
  {
    unsigned long long it = 0;
    while (!mbar_try_wait(bar, 0)) {
      if (++it > TMA_WAIT_LIMIT) {
        ok = false;
        break;
      }
    }
  }
  if (!ok) {
    if (a.status) atomicOr(a.status, 1);
    unsigned long long it = 0;  // let the copies land before the CTA's shared memory is released
    while (!mbar_try_wait(bar, 0) && ++it < TMA_WAIT_LIMIT) {
    }
    return;
  }

  float2 acc[24];
#pragma unroll
  for (int r = 0; r < 24; ++r) acc[r] = make_float2(0.f, 0.f);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      const bool fwd = dir == 0;
      const char* blk;
      const char* lnk;
      int ph = 1;
      if (mu == 0) {
        int xn = fwd ? c[0] + 1 : c[0] - 1;
        if (xn == g.L[0]) {
          xn = 0;
          ph = g.bc[0];
        } else if (xn < 0) {
          xn = g.L[0] - 1;
          ph = g.bc[0];
        }
        int b = (xn >> 1) - a0 + 1;  // position in the x range (a0 - 1 ... a0 + seg)
        if (b < 0) b += g.Lxh;
        if (b >= g.Lxh) b -= g.Lxh;
        blk = reinterpret_cast<const char*>(smem_raw + pl.off_x + (unsigned)b * pl.site_bytes);
        lnk = fwd ? reinterpret_cast<const char*>(smem_raw + pl.off_lfwd + (unsigned)sl * pl.lrow_bytes)
                  : reinterpret_cast<const char*>(smem_raw + pl.off_lbx + (unsigned)b * pl.lrow_bytes);
      } else {
        const int L = g.L[mu];
        if (fwd && c[mu] == L - 1) ph = g.bc[mu];
        if (!fwd && c[mu] == 0) ph = g.bc[mu];
        const int k = 2 * (mu - 1) + (fwd ? 0 : 1);
        blk = reinterpret_cast<const char*>(smem_raw + pl.off_rows + (unsigned)(k * seg + sl) * pl.site_bytes);
        lnk = fwd ? reinterpret_cast<const char*>(smem_raw + pl.off_lfwd + (unsigned)sl * pl.lrow_bytes)
                  : reinterpret_cast<const char*>(smem_raw + pl.off_lbr +
                                                  (unsigned)((mu - 1) * seg + sl) * pl.lrow_bytes);
      }
      float u[18];
      load_link_smem<P, C12>(lnk + mu * LB, u);
      float2 psi[24], h[12], uh[12];
      load_pair<P, Lsh, false>(blk, q, Lsh, psi);
      const float scale = ph < 0 ? -alpha : alpha;
      if (fwd) {
        project2<SF>(mu, psi, h);
        su3_mul2<false>(u, h, uh);
        accumulate2<SF>(mu, uh, scale, acc);
      } else {
        project2<-SF>(mu, psi, h);
        su3_mul2<true>(u, h, uh);
        accumulate2<-SF>(mu, uh, scale, acc);
      }
    }
  }

  // ------------------------------------------------------------ epilogue (as in dhop_body_pair)
  const size_t gsite_bytes = (size_t)Lsh * 2 * 24 * sizeof(T);
  char* outb = static_cast<char*>(a.out) + (size_t)site * gsite_bytes;
  if (a.pre != PRE_NONE) {
    const char* auxb = static_cast<const char*>(a.aux) + (size_t)site * gsite_bytes;
    const float2 B = f2((float)a.beta);
    if (a.pre == PRE_AUX) {
      float2 o[24];
      load_pair<P, Lsh>(auxb, q, Lsh, o);
#pragma unroll
      for (int r = 0; r < 24; ++r) acc[r] = ffma2(B, o[r], acc[r]);
    } else {
      float o0[24], o1[24];
      if (a.pre == PRE_MOOEE) {
        mooee_slice<P, false>(auxb, 2 * q, Ls, Lsh, a.d5, a.mass, o0);
        mooee_slice<P, false>(auxb, 2 * q + 1, Ls, Lsh, a.d5, a.mass, o1);
      } else {
        mooee_slice<P, true>(auxb, 2 * q, Ls, Lsh, a.d5, a.mass, o0);
        mooee_slice<P, true>(auxb, 2 * q + 1, Ls, Lsh, a.d5, a.mass, o1);
      }
#pragma unroll
      for (int r = 0; r < 24; ++r) acc[r] = ffma2(B, make_float2(o0[r], o1[r]), acc[r]);
    }
  }
  const bool pad_lane = (Ls & 1) && q == Lsh - 1;
  if (a.post == POST_NONE) {
    if (pad_lane) {
#pragma unroll
      for (int r = 0; r < 24; ++r) acc[r].y = 0.f;
    }
    store_pair<P, Lsh>(outb, q, Lsh, acc);
    return;
  }
  __syncthreads();  // all hops done: the staged buffers are free for the fifth-dimension solve
  float* sm = reinterpret_cast<float*>(smem_raw);
  {
    float* d0 = sm + ((size_t)sl * Ls + 2 * q) * 24;
#pragma unroll
    for (int r = 0; r < 24; ++r) d0[r] = acc[r].x;
    if (!pad_lane) {
#pragma unroll
      for (int r = 0; r < 24; ++r) d0[24 + r] = acc[r].y;
    }
  }
  __syncthreads();
  for (int task = tid; task < seg * 24; task += blockDim.x) {
    const int qq = task / 24;
    const int r = task - qq * 24;
    const bool upper = r < 12;
    const bool forward_form = (a.post == POST_INV) ? upper : !upper;
    mooee_inv_line<float>(sm + (size_t)qq * Ls * 24 + r, Ls, forward_form, (float)a.mass, (float)a.inv_d5,
                          (float)a.inv_den);
  }
  __syncthreads();
  const float* s0 = sm + ((size_t)sl * Ls + 2 * q) * 24;
#pragma unroll
  for (int r = 0; r < 24; ++r) acc[r] = make_float2(s0[r], pad_lane ? 0.f : s0[24 + r]);
  store_pair<P, Lsh>(outb, q, Lsh, acc);
}

template <int P, bool DAG, bool C12, int LSC>
__global__ void __launch_bounds__(256, 2) dhop_tma_kernel(const __grid_constant__ DhopArgs a) {
  dhop_tma_body<P, DAG, C12, LSC>(a);
}

// Largest segment (divisor of Lx/2, at most 16 sites and 256 threads) whose staged data fits two
// CTAs per SM; 0 when no segment qualifies (the direct kernel is used then).
inline int tma_choose_seg(int lxh, int Ls, int real_bytes, bool c12, size_t post_smem_per_site) {
  const int lb = link_bytes(real_bytes, c12);
  for (int seg = 16; seg >= 4; --seg) {
    if (lxh % seg || seg * ls_half(Ls) > 256) continue;
    const TmaPlan p = tma_plan(seg, Ls, real_bytes, lb);
    if (p.bytes > 110 * 1024) continue;
    if (post_smem_per_site * seg > p.bytes - 16) continue;
    return seg;
  }
  return 0;
}

}  // namespace gdwf
