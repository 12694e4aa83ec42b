// Radial transforms of the mixed-precision H X on the tensor cores (Algorithms 1 and 3).
//
// Per |n| group g the radial transforms are contractions of depth K (inverse) and N_r
// (forward) with one real table ξ_g shared by all (column, pair) items of the group:
//   inverse  G[c][p][a] = sum_k ξ_g[p][k] X[c][off(a) + k]              (k < Ka(a))
//   forward  Y[c][off(a) + k] = d x + sum_p O_g[k][p] H[c][p][a]        (k < Ka(a))
// With the items on the MMA's M dimension (128 rows = 64 items x {re, im}) both become
//   D[(item, part)][j] = sum_i A[(item, part)][i] B[j][i]
// with A the gathered coefficients (inverse: X rows over k; forward: H rows over p, in
// chunks of 32 radial nodes) and B the table (inverse: ξ_g rows p; forward: O_g rows k).
// Both operands are split into three BF16 parts, x = b0 + b1 + b2 (24 significant bits: the
// FP32 value exactly), and the products taken as the six part pairs (p, q) with p + q <= 2 by
// tcgen05 kind::f16 MMAs with FP32 accumulation in TMEM: the accuracy of the FP32 transforms.
// The tables are split once at setup and brought into shared memory by one TMA copy per K
// block (cp.async.bulk.tensor, 64-byte swizzle), which overlaps the staging of the other
// operand; the coefficients are split while they are staged into
// shared memory (K-major rows of 32 BF16, 64-byte swizzle), their global loads issued
// together before any is used.  The epilogue reads TMEM with one thread per (item, part) row: the inverse writes G
// rows of consecutive pairs (coalesced), the forward stages Y in shared memory and scatters it
// as the FP32 SIMT kernel does (diagonal term in FP64, the fused Chebyshev step).
// Every wait on an mbarrier is bounded; a wait that runs out sets HW_ETIMEOUT in the context's
// status word and the CTA skips its stores.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "hw_common.cuh"
#include "hw_ctx.h"
#include "hw_tc.cuh"

namespace hw {

constexpr int RT_ITEMS = 64;        // (column, pair) items per CTA: 128 MMA rows
constexpr int RT_THREADS = 256;

struct RadTcArgs {
  int Nr, K, nA, ncols, ns, c0;
  int npad;                 // inverse: N of the MMA = Nr rounded up to 16 (table rows)
  int kb;                   // inverse: K blocks of 32
  int kpad;                 // forward: N of the MMA = K rounded up to 16 (table rows)
  int kbp;                  // forward: N_r blocks of 32
  const int* group_start;
  const int* off;
  const int* Ka;
  int64_t ld;
  const double* ke;
  int64_t keoff[MAXSLOT];
  int step;
  ChebStep cs;
  int scale_mode;           // inverse: coefficients times i 2 pi m (1) or i 2 pi n Ncyc (2)
  const int* pair_n;
  const int* pair_mrow;
  const int* mrow_m;
  int ncyc;
  float2* gh;               // G (inverse output) or H (forward input)
  Blocks blk;
  int* status;
};

constexpr int RT_PLANES = 3;        // BF16 parts of every operand
constexpr int RT_ROWB = 64;         // bytes per K-major row: 32 BF16
constexpr int RT_ATILE = RT_PLANES * 128 * RT_ROWB;   // one K block of A, all parts

// one thread: the TMA copies of group g's table, K block kb to [kb][3][rows][64 B] (the three
// parts of a block are one box), completing on bar
__device__ __forceinline__ void load_table_tma(const CUtensorMap* map, int g, int rows, int kblocks,
                                               unsigned char* dst, uint64_t* bar) {
  mbar_expect_tx(bar, (uint32_t)(kblocks * RT_PLANES * rows * RT_ROWB));
  for (int kb = 0; kb < kblocks; ++kb)
    tma_load_3d(dst + (size_t)kb * RT_PLANES * rows * RT_ROWB, map, kb * 32, 0, g * RT_PLANES, bar);
}

// the six part products of one 32-element K block (two K steps of 16), A_p B_q with p + q <= 2:
// the leading product A_0 B_0 into the accumulator at column t0, the five smaller ones (2^-8
// and 2^-16 of it) into a second one at t1, so that the tensor core's accumulation does not
// round them against the leading terms; the epilogue adds the two
__device__ __forceinline__ void mma_bf16x3(uint32_t t0, uint32_t t1, uint32_t aBase, uint32_t bBase, int brows,
                                           uint32_t idesc, bool first) {
  const uint32_t aStride = 128 * RT_ROWB, bStride = (uint32_t)(brows * RT_ROWB);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const uint64_t o = (uint64_t)(s * 2);
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      const int pa = t < 3 ? (t == 2 ? 1 : 0) : (t == 3 ? 0 : (t == 4 ? 1 : 2));
      const int pb = t < 3 ? (t == 1 ? 1 : 0) : (t == 3 ? 2 : (t == 4 ? 1 : 0));
      const bool lead = t == 0;
      umma_bf16(lead ? t0 : t1, umma_desc<64>(aBase + pa * aStride) + o, umma_desc<64>(bBase + pb * bStride) + o,
                idesc, (first && s == 0 && (t == 0 || t == 1)) ? 0u : 1u);
    }
  }
}

// store the three BF16 parts of x at (row, col) of the three part planes of a K block
__device__ __forceinline__ void put3(unsigned char* tile, int row, int col, float x) {
  __nv_bfloat16 b0, b1, b2;
  bf16x3_split(x, b0, b1, b2);
  const uint32_t o = sw64_off(row, col);
  *reinterpret_cast<__nv_bfloat16*>(tile + o) = b0;
  *reinterpret_cast<__nv_bfloat16*>(tile + 128 * RT_ROWB + o) = b1;
  *reinterpret_cast<__nv_bfloat16*>(tile + 2 * 128 * RT_ROWB + o) = b2;
}

// ------------------------------------------------------------------------------- inverse
// grid: x = tile of RT_ITEMS items within group g, y = g.  Nine warps: warps 0-7 gather the
// coefficients and drain TMEM, warp 8 allocates TMEM and issues the MMAs.  A CTA of a kernel that
// allocates TMEM holds the SM's allocation permit until it has allocated: no further CTA of the
// kernel starts on that SM meanwhile.  So the allocation comes first, in its own warp, and the
// third CTA of an SM (two hold their 2 N_r columns at once) gathers while that warp waits for a
// sibling's columns.  Before griddep_wait only the basis's constant tables are read, and no TMEM
// is allocated.
constexpr int RI_THREADS = RT_THREADS + 32;
constexpr int RI_MMA_WARP = RT_THREADS / 32;
__global__ void __launch_bounds__(RI_THREADS, 3) k_rinv_tc(const __grid_constant__ CUtensorMap tmT, RadTcArgs A) {
  extern __shared__ __align__(1024) unsigned char rsm_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)rsm_raw + 1023) & ~(uintptr_t)1023);
  const int g = blockIdx.y;
  const int gs = A.group_start[g], na = A.group_start[g + 1] - gs;
  const long nitems = (long)na * A.ncols;
  const long q0 = (long)blockIdx.x * RT_ITEMS;
  if (na == 0 || q0 >= nitems) return;
  const int KB = A.kb, NP = A.npad;
  unsigned char* sA = sm;                                   // [KB][3][128][64 B]
  unsigned char* sB = sm + (size_t)KB * RT_ATILE;           // [KB][3][NP][64 B]
  __shared__ __align__(8) uint64_t bar_mma, bar_tab;
  __shared__ uint32_t tmem_s;
  __shared__ const double* s_x[RT_ITEMS];
  __shared__ float2* s_g[RT_ITEMS];
  __shared__ int s_ka[RT_ITEMS];
  __shared__ float s_sc[RT_ITEMS];
  __shared__ int s_tab_ok;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool mw = warp == RI_MMA_WARP;
  const uint32_t tcols = 2 * NP <= 32 ? 32 : (2 * NP <= 64 ? 64 : (2 * NP <= 128 ? 128 : (2 * NP <= 256 ? 256 : 512)));
  if (mw) {
    if (lane == 0) {
      mbar_init(&bar_mma, 1);
      mbar_init(&bar_tab, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      load_table_tma(&tmT, g, NP, KB, sB, &bar_tab);
    }
    __syncwarp();
    griddep_wait();
    tmem_alloc(&tmem_s, tcols);
  } else {
    if (threadIdx.x < RT_ITEMS) {
      const int q = threadIdx.x;
      const long item = q0 + q;
      const double* xp = nullptr;
      float2* gp = nullptr;
      int ka = 0;
      float sc = 0.f;
      if (item < nitems) {
        const int c = (int)(item / na), a = gs + (int)(item - (long)c * na);
        const int cg = A.c0 + c;
        const int slot = cg / A.ns, sl = cg - slot * A.ns;
        const int kbk = A.blk.kb[slot];
        ka = A.Ka[(size_t)kbk * A.nA + a];
        xp = A.blk.x[slot] + 2 * ((size_t)A.off[(size_t)kbk * A.nA + a] + (size_t)sl * A.ld);
        gp = A.gh + (size_t)c * A.Nr * A.nA + a;
        if (A.scale_mode != 0)
          sc = (float)(6.283185307179586 * (A.scale_mode == 1 ? (double)A.mrow_m[A.pair_mrow[a]]
                                                               : (double)A.pair_n[a] * A.ncyc));
      }
      s_x[q] = xp;
      s_g[q] = gp;
      s_ka[q] = ka;
      s_sc[q] = sc;
    }
    griddep_wait();   // X is the previous kernels' output
    asm volatile("bar.sync 1, %0;" ::"r"(RT_THREADS) : "memory");   // the gather warps only
    // A rows (2q + part) over k: a warp takes the items warp, warp + 8, ...; lanes over k.  Every
    // load of the warp's items is issued before the first is used.
    constexpr int IW = RT_ITEMS / (RT_THREADS / 32);   // items per warp
    for (int kb = 0; kb < KB; ++kb) {
      const int k = kb * 32 + lane;
      double xr[IW], xi[IW];
#pragma unroll
      for (int i = 0; i < IW; ++i) {
        const int q = warp + 8 * i;
        xr[i] = 0.0;
        xi[i] = 0.0;
        if (k < s_ka[q]) {
          xr[i] = s_x[q][2 * k];
          xi[i] = s_x[q][2 * k + 1];
        }
      }
      unsigned char* tile = sA + (size_t)kb * RT_ATILE;
#pragma unroll
      for (int i = 0; i < IW; ++i) {
        const int q = warp + 8 * i;
        float re = d2f(xr[i]), im = d2f(xi[i]);
        if (A.scale_mode != 0) {   // times i s
          const float sc = s_sc[q], t = re;
          re = -sc * im;
          im = sc * t;
        }
        put3(tile, 2 * q, lane, re);
        put3(tile, 2 * q + 1, lane, im);
      }
    }
    fence_proxy_async();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_s;
  if (mw && lane == 0) {
    s_tab_ok = mbar_wait(&bar_tab, 0);
    if (s_tab_ok) {
      const uint32_t idesc = umma_idesc_bf16(NP);
      for (int kb = 0; kb < KB; ++kb)
        mma_bf16x3(tmem, tmem + (uint32_t)NP, smem_u32(sA + (size_t)kb * RT_ATILE),
                   smem_u32(sB + (size_t)kb * RT_PLANES * NP * RT_ROWB), NP, idesc, kb == 0);
      umma_commit(&bar_mma);
    } else {
      atomicExch(A.status, HW_ETIMEOUT);
    }
  }
  __syncthreads();
  const bool tab_ok = s_tab_ok;
  bool ok = tab_ok && mbar_wait(&bar_mma, 0);
  griddep_launch();   // only the drain is left: the next kernel's CTAs may start
  if (!ok && threadIdx.x == 0) atomicExch(A.status, HW_ETIMEOUT);
  tc_fence_after();
  if (ok && !mw) {
    // lane quadrant = warp % 4: row 2q + part holds D[row][p] for all p; warps w and w + 4 take
    // alternate 16-column chunks.  The lanes of an item's re and im rows swap halves so that
    // each stores one complex entry per column pair: the re lane column p, the im lane p + 1.
    const int quad = warp & 3, half = warp >> 2;
    const int row = quad * 32 + lane, q = row >> 1, part = row & 1;
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
    float2* gp = s_g[q];
    for (int p0 = 16 * half; p0 < NP; p0 += 32) {
      uint32_t v[16], u[16];
      tmem_ld16(tl + (uint32_t)p0, v);
      tmem_ld16(tl + (uint32_t)(NP + p0), u);
#pragma unroll
      for (int j = 0; j < 16; j += 2) {
        const float a0 = __uint_as_float(v[j]) + __uint_as_float(u[j]);           // this part, column p0 + j
        const float a1 = __uint_as_float(v[j + 1]) + __uint_as_float(u[j + 1]);   // column p0 + j + 1
        const float got = __shfl_xor_sync(0xffffffffu, part ? a0 : a1, 1);
        const int p = p0 + j + part;
        if (gp && p < A.Nr) gp[(size_t)p * A.nA] = part ? make_float2(got, a1) : make_float2(a0, got);
      }
    }
  }
  if (!ok && tab_ok) {   // the tensor core must be done with TMEM before it is released
    if (!mbar_wait(&bar_mma, 0) && threadIdx.x == 0) atomicExch(A.status, HW_ETIMEOUT);
  }
  if (!tab_ok && mw && lane == 0) mbar_wait(&bar_tab, 0);   // the copies in flight land before exit
  tc_fence_before();
  __syncthreads();
  if (mw) {
    tc_fence_after();
    tmem_dealloc(tmem, tcols);
  }
}

// ------------------------------------------------------------------------------- forward
// grid: x = tile of RT_ITEMS items within group g, y = g.  No nu != 0 terms (the SIMT kernel
// takes those launches).  Before griddep_wait only the basis's constant tables are read.  TMEM
// (2 K_p columns, three CTAs per SM within the 512) is allocated first, so that the SM's
// allocation permit passes on at once and all three CTAs start while the slab drains: the kernel
// before this one is always a slab kernel, which holds no TMEM, and that kernel signals its
// dependents only after its own wait, so every earlier kernel has completed when a CTA of this
// one starts.
__global__ void __launch_bounds__(RT_THREADS, 3) k_rfwd_tc(const __grid_constant__ CUtensorMap tmT, RadTcArgs A) {
  extern __shared__ __align__(1024) unsigned char rsm_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)rsm_raw + 1023) & ~(uintptr_t)1023);
  const int g = blockIdx.y;
  const int gs = A.group_start[g], na = A.group_start[g + 1] - gs;
  const long nitems = (long)na * A.ncols;
  const long q0 = (long)blockIdx.x * RT_ITEMS;
  if (na == 0 || q0 >= nitems) return;
  const int KBP = A.kbp, KP = A.kpad, K = A.K, Nr = A.Nr;
  unsigned char* sA = sm;                                   // 2 stages x [3][128][64 B]
  unsigned char* sB = sm + 2 * RT_ATILE;                    // [KBP][3][KP][64 B]
  float2* Ys = reinterpret_cast<float2*>(sm);               // [RT_ITEMS][K + 1], after the MMAs
  __shared__ __align__(8) uint64_t bar_mma[2], bar_tab;
  __shared__ uint32_t tmem_s;
  __shared__ const float2* s_h[RT_ITEMS];
  __shared__ int64_t s_o[RT_ITEMS], s_cs[RT_ITEMS];
  __shared__ int s_ka[RT_ITEMS], s_slot[RT_ITEMS];
  __shared__ int s_bad;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t tcols = 2 * KP <= 32 ? 32 : (2 * KP <= 64 ? 64 : (2 * KP <= 128 ? 128 : (2 * KP <= 256 ? 256 : 512)));
  if (threadIdx.x == 0) {
    mbar_init(&bar_mma[0], 1);
    mbar_init(&bar_mma[1], 1);
    mbar_init(&bar_tab, 1);
    s_bad = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    load_table_tma(&tmT, g, KP, KBP, sB, &bar_tab);
  }
  if (warp == 0) tmem_alloc(&tmem_s, tcols);
  if (threadIdx.x < RT_ITEMS) {
    const int qq = threadIdx.x;
    const long it = q0 + qq;
    const float2* hp = nullptr;
    int64_t o = 0, cs = 0;
    int ka = 0, slot = 0;
    if (it < nitems) {
      const int cc = (int)(it / na), aa = gs + (int)(it - (long)cc * na);
      const int cg = A.c0 + cc;
      slot = cg / A.ns;
      const int sl = cg - slot * A.ns;
      const int kb = A.blk.kb[slot];
      ka = A.Ka[(size_t)kb * A.nA + aa];
      o = (int64_t)A.off[(size_t)kb * A.nA + aa];
      cs = (int64_t)sl * A.ld;
      hp = A.gh + (size_t)cc * Nr * A.nA + aa;
    }
    s_h[qq] = hp;
    s_o[qq] = o;
    s_cs[qq] = cs;
    s_ka[qq] = ka;
    s_slot[qq] = slot;
  }
  griddep_wait();   // H, X and Y are the previous kernels' data
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_s;
  const uint32_t idesc = umma_idesc_bf16(KP);
  // a warp fills 8 items x 4 radial nodes per step (64-byte segments of H rows in global
  // memory); its eight steps' loads are issued before the first is used
  const int li = lane & 7, lp = lane >> 3;
  for (int j = 0; j < KBP; ++j) {
    const int st = j & 1;
    unsigned char* tile = sA + (size_t)st * RT_ATILE;
    float2 h[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {   // the loads first: they overlap the wait for the stage
      const int t = warp + 8 * i;
      const int q = (t & 7) * 8 + li, p = j * 32 + (t >> 3) * 4 + lp;
      const float2* hp = s_h[q];
      h[i] = (hp && p < Nr) ? hp[(size_t)p * A.nA] : make_float2(0.f, 0.f);
    }
    if (j >= 2 && !mbar_wait(&bar_mma[st], (uint32_t)(((j - 2) >> 1) & 1))) s_bad = 1;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int t = warp + 8 * i;
      const int q = (t & 7) * 8 + li, pl = (t >> 3) * 4 + lp;
      put3(tile, 2 * q, pl, h[i].x);
      put3(tile, 2 * q + 1, pl, h[i].y);
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0 && j == 0 && !mbar_wait(&bar_tab, 0)) s_bad = 2;   // the table is in
    if (threadIdx.x == 0 && !s_bad) {
      mma_bf16x3(tmem, tmem + (uint32_t)KP, smem_u32(tile), smem_u32(sB + (size_t)j * RT_PLANES * KP * RT_ROWB), KP,
                 idesc, j == 0);
      umma_commit(&bar_mma[st]);
    }
  }
  // the last chunk's MMAs (and with them all earlier ones) complete
  const int jl = KBP - 1;
  __syncthreads();   // s_bad as the MMA thread left it
  const int bad = s_bad;
  bool ok = !bad && mbar_wait(&bar_mma[jl & 1], (uint32_t)((jl >> 1) & 1));
  griddep_launch();   // only the drain and the output are left: the next kernel's CTAs may start
  if (!ok && threadIdx.x == 0) atomicExch(A.status, HW_ETIMEOUT);
  tc_fence_after();
  __syncthreads();   // every thread is past its reads of the A stages (Ys reuses them)
  if (ok) {   // lane quadrant = warp % 4; warps w and w + 4 take alternate 16-column chunks
    const int quad = warp & 3, half = warp >> 2;
    const int row = quad * 32 + lane, q = row >> 1, part = row & 1;
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
    for (int k0 = 16 * half; k0 < KP; k0 += 32) {
      uint32_t v[16], u[16];
      tmem_ld16(tl + (uint32_t)k0, v);
      tmem_ld16(tl + (uint32_t)(KP + k0), u);
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const int k = k0 + jj;
        if (k < K)
          reinterpret_cast<float*>(&Ys[q * (K + 1) + k])[part] = __uint_as_float(v[jj]) + __uint_as_float(u[jj]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (ok) {
#pragma unroll 4
    for (int idx = threadIdx.x; idx < RT_ITEMS * K; idx += RT_THREADS) {
      const int qq = idx / K, k = idx - qq * K;
      if (k >= s_ka[qq]) continue;
      const int slot = s_slot[qq];
      const int64_t o = s_o[qq] + k;
      const double* x = A.blk.x[slot] + 2 * (o + s_cs[qq]);
      double* y = A.blk.y[slot] + 2 * (o + s_cs[qq]);
      const double d = A.ke[A.keoff[slot] + o];
      const float2 hv = Ys[qq * (K + 1) + k];
      const double x0 = x[0], x1 = x[1];
      double y0 = d * x0 + double(hv.x), y1 = d * x1 + double(hv.y);
      if (A.step) {
        const double al = A.cs.al[slot], c2 = A.cs.c[slot], be = A.cs.be[slot];
        y0 = al * (y0 - c2 * x0);
        y1 = al * (y1 - c2 * x1);
        if (be != 0.0) {
          y0 -= be * y[0];
          y1 -= be * y[1];
        }
      }
      y[0] = y0;
      y[1] = y1;
    }
  } else if (bad != 2) {   // the tensor core must be done with TMEM before it is released
    if (!mbar_wait(&bar_mma[jl & 1], (uint32_t)((jl >> 1) & 1)) && threadIdx.x == 0)
      atomicExch(A.status, HW_ETIMEOUT);
  } else if (threadIdx.x == 0) {   // no MMA issued; the table copies land before exit
    mbar_wait(&bar_tab, 0);
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, tcols);
  }
}

// ------------------------------------------------------------------------------- host
size_t rinv_tc_smem(int npad, int kb) { return (size_t)kb * RT_PLANES * (128 + npad) * RT_ROWB + 1024; }
size_t rfwd_tc_smem(int kpad, int kbp) {
  return (size_t)2 * RT_ATILE + (size_t)kbp * RT_PLANES * kpad * RT_ROWB + 1024;
}

// Split table of one direction: src [(N+1)][rows_src][cols_src] FP64, element (r, c) at
// r * cols_src + c, into [(N+1)][3][rows][cblocks*32] BF16 parts b0 + b1 + b2 (24 bits),
// zero-padded.
static void split_table(const std::vector<double>& src, int ngroups, int rows_src, int cols_src, int rows,
                        int cblocks, std::vector<__nv_bfloat16>& out) {
  auto bf = [](double x) {   // round to BF16 (through FP32), returned with its value
    const float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    float r;
    memcpy(&r, &u, 4);
    return r;
  };
  const int cw = cblocks * 32;
  out.assign((size_t)ngroups * RT_PLANES * rows * cw, __float2bfloat16_rn(0.f));
  for (int gi = 0; gi < ngroups; ++gi)
    for (int r = 0; r < rows_src; ++r)
      for (int c = 0; c < cols_src; ++c) {
        double x = src[((size_t)gi * rows_src + r) * cols_src + c];
        for (int pl = 0; pl < RT_PLANES; ++pl) {
          const float b = bf(x);
          out[(((size_t)gi * RT_PLANES + pl) * rows + r) * cw + c] = __float2bfloat16_rn(b);
          x -= (double)b;
        }
      }
}

cudaError_t radial_tc_setup(hw_ctx* ctx, const HostBasis& hb, const std::vector<double>& rinv,
                            const std::vector<double>& rfwd) {
  auto& db = ctx->db;
  const int Nr = hb.prm.Nr, K = hb.K, G = hb.N + 1;
  db.rt_npad = (Nr + 15) / 16 * 16;
  db.rt_kb = (K + 31) / 32;
  db.rt_kpad = (K + 15) / 16 * 16;
  db.rt_kbp = (Nr + 31) / 32;
  db.rt_ok = db.rt_npad <= 256 && db.rt_kpad <= 256 && db.rt_kb <= 2 &&
             rinv_tc_smem(db.rt_npad, db.rt_kb) <= 227 * 1024 && rfwd_tc_smem(db.rt_kpad, db.rt_kbp) <= 227 * 1024;
  if (!db.rt_ok) return cudaSuccess;
  std::vector<__nv_bfloat16> ti, tf;
  split_table(rinv, G, Nr, K, db.rt_npad, db.rt_kb, ti);     // rows p, columns k
  split_table(rfwd, G, K, Nr, db.rt_kpad, db.rt_kbp, tf);    // rows k, columns p
  cudaError_t e = cudaMalloc((void**)&db.rt_inv, ti.size() * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMemcpy(db.rt_inv, ti.data(), ti.size() * 2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)&db.rt_fwd, tf.size() * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMemcpy(db.rt_fwd, tf.data(), tf.size() * 2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess &&
      !(make_plane_map(&db.rt_map_inv, db.rt_inv, false, (int64_t)db.rt_kb * 32, db.rt_npad, G * RT_PLANES,
                       db.rt_npad, RT_PLANES, 64) &&
        make_plane_map(&db.rt_map_fwd, db.rt_fwd, false, (int64_t)db.rt_kbp * 32, db.rt_kpad, G * RT_PLANES,
                       db.rt_kpad, RT_PLANES, 64))) {
    db.rt_ok = false;   // no TMA map: the SIMT kernels take the launches
    return cudaSuccess;
  }
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rinv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)rinv_tc_smem(db.rt_npad, db.rt_kb));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rfwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)rfwd_tc_smem(db.rt_kpad, db.rt_kbp));
  // the largest shared-memory carveout: without it the driver's choice held two inverse CTAs per
  // SM, and the third of an SM started only when one of the first two had finished
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rinv_tc, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rfwd_tc, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  return e;
}

static RadTcArgs tc_args(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld, int nc, int c0, void* gh) {
  auto& hb = ctx->hb;
  auto& db = ctx->db;
  RadTcArgs a;
  a.Nr = hb.prm.Nr;
  a.K = hb.K;
  a.nA = hb.nA;
  a.ncols = nc;
  a.ns = ns;
  a.c0 = c0;
  a.npad = db.rt_npad;
  a.kb = db.rt_kb;
  a.kpad = db.rt_kpad;
  a.kbp = db.rt_kbp;
  a.group_start = db.group_start;
  a.off = db.off;
  a.Ka = db.Ka;
  a.ld = ld;
  a.ke = db.ke;
  for (int i = 0; i < blk.nslot; ++i) a.keoff[i] = db.ke_off[blk.kb[i]];
  a.step = 0;
  a.scale_mode = 0;
  a.pair_n = db.pair_n;
  a.pair_mrow = db.pair_mrow;
  a.mrow_m = db.mrow_m;
  a.ncyc = hb.prm.ncyc;
  a.gh = reinterpret_cast<float2*>(gh);
  a.blk = blk;
  a.status = ctx->dflag;
  return a;
}

static dim3 tc_grid(const hw_ctx* ctx, int nc) {
  const auto& hb = ctx->hb;
  int maxna = 0;
  for (int g = 0; g <= hb.N; ++g) maxna = std::max(maxna, hb.group_start[g + 1] - hb.group_start[g]);
  return dim3((unsigned)(((long)maxna * nc + RT_ITEMS - 1) / RT_ITEMS), hb.N + 1);
}

cudaError_t launch_rinv_tc(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld, int nc, int c0, void* gbuf,
                           int scale_mode) {
  RadTcArgs a = tc_args(ctx, blk, ns, ld, nc, c0, gbuf);
  a.scale_mode = scale_mode;
  return launch_ex(ctx, ctx->overlap_launch != 0, k_rinv_tc, tc_grid(ctx, nc), dim3(RI_THREADS),
                   rinv_tc_smem(a.npad, a.kb), ctx->db.rt_map_inv, a);
}

cudaError_t launch_rfwd_tc(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld, int nc, int c0, void* hbuf,
                           const ChebStep* step) {
  RadTcArgs a = tc_args(ctx, blk, ns, ld, nc, c0, hbuf);
  if (step) {
    a.step = 1;
    a.cs = *step;
  }
  return launch_ex(ctx, ctx->overlap_launch != 0, k_rfwd_tc, tc_grid(ctx, nc), dim3(RT_THREADS),
                   rfwd_tc_smem(a.kpad, a.kbp), ctx->db.rt_map_fwd, a);
}

}  // namespace hw
