// The GEMM family the stage-centric model of arxiv 2605.04178 predicts
// (Sec. III-A, Fig. "cta-exec-model"): per K-step a TMA load of the A and B
// tiles into a shared-memory ring (Eq. 4), tcgen05.mma into an FP32 TMEM
// accumulator (Eqs. 2-3; Eq. 6 for CTA pairs), mbarrier hand-offs (T_sync),
// and an epilogue that drains TMEM to global memory (T_store).
//
// Kernel shape (sm_103a): one persistent CTA per SM (CTA pair per two SMs for
// cta_group 2), 6 warps:
//   warp 0      TMA producer (one thread): waits empty[s], loads stage s;
//   warp 1      TMEM allocator and MMA issuer: the whole warp runs the
//               K-loop (waits full[s], forms the descriptors) and one lane
//               issues BK/k_instr MMAs per row block and commits to
//               empty[s]; after the last K-step it commits to acc_full[buffer];
//   warps 2..5  epilogue: wait acc_full, tcgen05.ld 32-column chunks, scale,
//               store FP32 C (masked at the M/N edges), release the buffer.
// TMEM strategy A keeps only the accumulators in tensor memory and feeds both
// operands from shared memory; strategy B (one SM, 128-row blocks) first
// copies each A K-slice of the stage into tensor memory with tcgen05.cp and
// the MMAs read A from there (Sec. III-A.1, "two TMEM strategies").
// Two TMEM accumulator buffers when they fit, so the epilogue of tile i
// overlaps the main loop of tile i+1.  When one accumulator fills TMEM (two
// 128-row blocks of 256 columns) the two row blocks are released separately:
// tile i+1 starts on row block 0 while the epilogue still drains row block 1.  Each CTA of a pair loads its own A
// rows and half of B (traffic 2 M_A + M_B per pair, no multicast); the pair
// leader issues the cta_group::2 MMAs.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdlib.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "pm_internal.cuh"

namespace pm {

constexpr int kGemmThreads = 192;
constexpr int kMaxStages = 6;
constexpr int kRasterGroup = 8;

constexpr int kMaxGroups = 128;

// Problems of one launch.  A single GEMM is one group.  Tiles are listed
// group by group (tile_off is the prefix sum); inside a group they are
// visited in bands of kRasterGroup (pair-)rows for L2 reuse.  A launch of
// several groups lists them largest tile (BM x BN) first and its CTAs (CTA
// pairs) take the tiles in alternating round-robin order (round_tile).
struct GroupTable {
  int n_groups;
  int tile_off[kMaxGroups + 1];
  int row0[kMaxGroups];        // first row of A_g / C_g in the stacked A / C
  int rows[kMaxGroups];        // M_g
  int brow0[kMaxGroups];       // first row of B_g (K-major) in the stacked B
  int tiles_m[kMaxGroups];     // row tiles (pair rows for cta_group 2)
  int tiles_n[kMaxGroups];
  uint8_t bm_idx[kMaxGroups];  // BM = 64 << bm_idx
  uint8_t bn_idx[kMaxGroups];  // BN = 64 << bn_idx
};

// TMA descriptors, one per box height in use: A boxes BM rows, B boxes BN/cta_group rows.
struct TensorMaps {
  CUtensorMap a[3];
  CUtensorMap b[3];
  CUtensorMap c;                   // FP32 C, 32 x 32 boxes, 128-byte swizzle (TMA-store epilogue)
};

struct GemmParams {
  int N, BK, stages, Kt;
  int sw;                          // swizzle span in bytes (64 or 128)
  int n_atoms;                     // swizzle atoms along K per stage
  int acc_cols, nbuf, alloc_cols;  // TMEM columns per accumulator buffer (largest tile)
  int split;                       // one buffer of two 128-row blocks, released block by block
  int a_col0, a_cols;              // strategy B: first TMEM column of the A ring, columns per stage
  uint32_t stage_bytes;            // ring stride (largest tile)
  uint32_t ab_fmt;                 // tcgen05 operand format code
  int lo_row_a, lo_row_b;          // row offset of the lo half (three-pass TF32)
  float* C;
  const float* scales;             // FP8: {s_A, s_B}
  int tma_store;                   // epilogue stages 32x32 chunks in shared memory and stores them by TMA
  uint32_t staging_off;            // byte offset of the epilogue staging area after the ring
  Watchdog wd;
};

// Position of the tile CTA (pair) `cta` of `n_ctas` runs in round r, or -1
// past the last tile.  One group: plain round-robin (round r holds tiles
// r*n_ctas .. r*n_ctas + n_ctas - 1, CTA c the c-th).  Several groups: the
// order is reversed on odd rounds, so the CTA that took the largest tile of
// a round takes the smallest of the next; with the groups listed largest
// tile first this evens out the CTAs' busy time like a longest-first
// schedule, and the stage model's grouped makespan follows the same rule.
__device__ __forceinline__ int round_tile(int r, int cta, int n_ctas, int n_tiles, bool snake) {
  const int t = r * n_ctas + ((snake && (r & 1)) ? n_ctas - 1 - cta : cta);
  return t < n_tiles ? t : -1;
}

// Everything the three roles need about one tile.
struct Tile {
  int arow, brow;                  // first operand rows this CTA loads
  int crow0, crow_end, ccol0;      // output rows [crow0, crow_end) capped by the group, first column
  int BM, BN, n_mblk, layout, ma, mb;
  uint32_t a_part, b_part, tx, idesc;
};

// q_hint: the group of this role's previous tile (0 at the start).  A
// role's tile positions only increase, so the search for the tile's group
// resumes there instead of scanning the table from its first group.
template <int CG, int L>
__device__ __forceinline__ void decode_tile(int t, const GemmParams& p, const GroupTable& g, uint32_t rank,
                                            Tile& T, int& q_hint) {
  int q = q_hint;
  while (q + 1 < g.n_groups && t >= g.tile_off[q + 1]) ++q;
  q_hint = q;
  const int lt = t - g.tile_off[q];
  const int tiles_n = g.tiles_n[q], tiles_m = g.tiles_m[q];
  const int per_band = kRasterGroup * tiles_n;
  const int band = lt / per_band;
  const int first = band * kRasterGroup;
  const int bsz = min(tiles_m - first, kRasterGroup);
  const int r = lt % per_band;
  const int tm = first + r % bsz, tn = r / bsz;
  T.ma = g.bm_idx[q];
  T.mb = g.bn_idx[q];
  T.BM = 64 << T.ma;
  T.BN = 64 << T.mb;
  T.arow = g.row0[q] + tm * CG * T.BM + (int)rank * T.BM;
  T.brow = g.brow0[q] + tn * T.BN + (int)rank * (T.BN / CG);
  T.crow0 = T.arow;
  T.crow_end = g.row0[q] + g.rows[q];
  T.ccol0 = tn * T.BN;
  T.n_mblk = (T.BM + 127) >> 7;
  // TMEM layout of the accumulator: 0 = one row per lane (128-row blocks);
  // 1 = 64 rows in lanes 0-15 of each 32-lane quarter (M = 64, one SM);
  // 2 = 64 rows in lanes 0-63 for columns [0, N/2) and again in lanes 64-127
  //     for columns [N/2, N) (M = 128 split over a CTA pair).
  T.layout = T.BM >= 128 ? 0 : (CG == 1 ? 1 : 2);
  T.a_part = (uint32_t)T.BM * p.sw;
  T.b_part = (uint32_t)(T.BN / CG) * p.sw;
  T.tx = (uint32_t)(L * p.n_atoms) * (T.a_part + T.b_part);
  const int mma_m = CG == 1 ? min(T.BM, 128) : 2 * min(T.BM, 128);
  T.idesc = instr_desc(p.ab_fmt, (uint32_t)mma_m, (uint32_t)T.BN);
}

// TMEM column (relative to the stage's A slot) of the 128 x 32-byte A slice
// (plane h, swizzle atom a, k-step kk, 128-row block m) under strategy B.
template <int NATOMS, int NK, int NMBLK>
__device__ __forceinline__ constexpr uint32_t ta_col(int h, int a, int kk, int m) {
  return 8u * (uint32_t)(((h * NATOMS + a) * NK + kk) * NMBLK + m);
}

// All MMAs of one pipeline stage, fully unrolled.  Descriptors are built once
// per stage; each MMA advances them by constant offsets (the start address
// sits in the low 14 bits in 16-byte units).  NATOMS swizzle atoms along K,
// NK = swizzle span / 32 B k-steps per atom, NMBLK 128-row blocks; three-pass
// TF32 adds the hi.lo and lo.hi products.  TA (strategy B): the stage's A
// slices are first copied to TMEM at a_tm and the MMAs read A from there.
template <int CG, int KIND, int NATOMS, int NK, int NMBLK, int TA>
__device__ __forceinline__ void issue_stage(uint32_t d0, uint64_t a0, uint64_t b0, uint32_t a_part16,
                                            uint32_t b_part16, uint32_t mblk16, uint32_t idesc, uint32_t bn,
                                            bool first, uint32_t a_tm, uint32_t issue) {
  constexpr int PASSES = (KIND == 1) ? 3 : 1;
  if constexpr (TA) {
    constexpr int L = (KIND == 1) ? 2 : 1;
#pragma unroll
    for (int h = 0; h < L; ++h)
#pragma unroll
      for (int a = 0; a < NATOMS; ++a)
#pragma unroll
        for (int kk = 0; kk < NK; ++kk)
#pragma unroll
          for (int m = 0; m < NMBLK; ++m)
            tmem_cp_128x256b(a_tm + ta_col<NATOMS, NK, NMBLK>(h, a, kk, m),
                             a0 + (uint64_t)((h * NATOMS + a) * a_part16 + m * mblk16 + 2u * kk), issue);
  }
#pragma unroll
  for (int pass = 0; pass < PASSES; ++pass) {
    const uint32_t ha = (pass == 2) ? 1u : 0u, hb = (pass == 1) ? 1u : 0u;
#pragma unroll
    for (int a = 0; a < NATOMS; ++a) {
#pragma unroll
      for (int kk = 0; kk < NK; ++kk) {
        const uint64_t bd = b0 + (uint64_t)((hb * NATOMS + a) * b_part16 + 2u * kk);
        const uint32_t acc = (first && pass == 0 && a == 0 && kk == 0) ? 0u : 1u;
#pragma unroll
        for (int m = 0; m < NMBLK; ++m) {
          if constexpr (TA) {
            umma_ta<KIND>(d0 + (uint32_t)m * bn, a_tm + ta_col<NATOMS, NK, NMBLK>(ha, a, kk, m), bd, idesc, acc,
                          issue);
          } else {
            const uint64_t ad = a0 + (uint64_t)((ha * NATOMS + a) * a_part16 + m * mblk16 + 2u * kk);
            umma<CG, KIND>(d0 + (uint32_t)m * bn, ad, bd, idesc, acc, issue);
          }
        }
      }
    }
  }
}

// Barriers and buffers the MMA issuer's K-loop works with.
struct MmaRing {
  uint64_t* full;
  uint64_t* empty;
  uint64_t* acce;
  int stage;
  uint32_t phase;
  uint32_t issue;                  // this lane issues the warp's tensor instructions
};

// A wait of the whole MMA warp: every lane waits, and the outcome is made
// warp-uniform so the warp leaves together if the watchdog gave up.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, const Watchdog& wd, volatile int* abort_p,
                                          unsigned site) {
  return __all_sync(0xffffffffu, mbar_wait(bar, parity, wd, abort_p, site)) != 0;
}

// One K-step's MMAs and the commit that frees its ring stage.
template <int CG, int KIND, int NA, int NK, int NM, int TA>
__device__ __forceinline__ void mma_step(MmaRing& r, const GemmParams& p, uint32_t d0, uint64_t a0, uint64_t b0,
                                         uint32_t a16, uint32_t b16, uint32_t m16, uint32_t idesc, uint32_t bn,
                                         bool first, uint32_t a_tm) {
  issue_stage<CG, KIND, NA, NK, NM, TA>(d0, a0, b0, a16, b16, m16, idesc, bn, first, a_tm, r.issue);
  if constexpr (CG == 1) umma_commit(smem_u32(&r.empty[r.stage]), r.issue);
  else umma_commit_pair(smem_u32(&r.empty[r.stage]), (uint16_t)3, r.issue);
  if (++r.stage == p.stages) { r.stage = 0; r.phase ^= 1u; }
}

// The MMA issuer's K-loop for one tile, specialised on the stage's shape
// (NA swizzle atoms along K, NK k-steps per atom, NM 128-row blocks) so the
// per-K-step path is a barrier wait, descriptor additions, the unrolled MMAs
// and a commit: the issuing thread is then never the bottleneck of the tensor
// pipe (a shape switch inside the loop cost a quarter of the throughput of
// four-MMA K-steps).  Under split release (256 x 256 tiles) the first K-step
// is peeled off; elsewhere it stays in the loop to keep the code small.
// Returns false if a wait gave up.
template <int CG, int KIND, int TA, int NA, int NK, int NM>
__device__ __forceinline__ bool mma_tile(MmaRing& r, const GemmParams& p, const Tile& T, uint32_t d0, uint32_t base,
                                         uint32_t tmem_base, uint32_t use, volatile int* abort_p) {
  constexpr int L = (KIND == 1) ? 2 : 1;
  const uint32_t swcode = p.sw == 128 ? 2u : 4u;
  const uint64_t desc0 = smem_desc(base, 8u * (uint32_t)p.sw, swcode);    // stage 0, first A atom
  const uint32_t stage16 = p.stage_bytes >> 4;                              // descriptor units (16 B)
  const uint32_t a16 = T.a_part >> 4, b16 = T.b_part >> 4, m16 = (uint32_t)(128 * p.sw) >> 4;
  const uint32_t boff16 = (uint32_t)(L * NA) * a16;                         // B follows the A atoms
  const uint32_t bn = (uint32_t)T.BN;
  int kt0 = 0;
  if constexpr (NM == 2 && !TA) {
    if (p.split) {
      // row block 0 now, row block 1 once the epilogue has drained it from
      // the previous tile
      if (!warp_wait(smem_u32(&r.full[r.stage]), r.phase, p.wd, abort_p, SITE_GEMM_MMA)) return false;
      tc_fence_after();
      const uint64_t a0 = desc0 + (uint64_t)((uint32_t)r.stage * stage16);
      const uint64_t b0 = a0 + (uint64_t)boff16;
      issue_stage<CG, KIND, NA, NK, 1, TA>(d0, a0, b0, a16, b16, m16, T.idesc, bn, true, 0u, r.issue);
      if (!warp_wait(smem_u32(&r.acce[1]), (use & 1u) ^ 1u, p.wd, abort_p, SITE_GEMM_MMA)) return false;
      tc_fence_after();
      mma_step<CG, KIND, NA, NK, 1, TA>(r, p, d0 + bn, a0 + (uint64_t)m16, b0, a16, b16, m16, T.idesc, bn, true, 0u);
      kt0 = 1;
    }
  }
  for (int kt = kt0; kt < p.Kt; ++kt) {
    if (!warp_wait(smem_u32(&r.full[r.stage]), r.phase, p.wd, abort_p, SITE_GEMM_MMA)) return false;
    tc_fence_after();
    const uint64_t a0 = desc0 + (uint64_t)((uint32_t)r.stage * stage16);
    const uint32_t a_tm = TA ? tmem_base + (uint32_t)(p.a_col0 + r.stage * p.a_cols) : 0u;
    mma_step<CG, KIND, NA, NK, NM, TA>(r, p, d0, a0, a0 + (uint64_t)boff16, a16, b16, m16, T.idesc, bn, kt == 0,
                                       a_tm);
  }
  return true;
}

template <int CG, int KIND, int TA>
__global__ void __launch_bounds__(kGemmThreads, 1)
    gemm_kernel(const __grid_constant__ TensorMaps maps, const __grid_constant__ GroupTable g,
                const GemmParams p) {
  extern __shared__ __align__(1024) uint8_t dsmem[];
  __shared__ __align__(8) uint64_t full_bar[kMaxStages];
  __shared__ __align__(8) uint64_t empty_bar[kMaxStages];
  __shared__ __align__(8) uint64_t accf_bar[2];
  __shared__ __align__(8) uint64_t acce_bar[2];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  constexpr int L = (KIND == 1) ? 2 : 1;              // operand halves (hi, lo) for three-pass TF32
  constexpr int E = (KIND == 0) ? 2 : (KIND == 1 ? 4 : 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = (CG == 2) ? cluster_ctarank() : 0u;
  const int cta = (CG == 2) ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int n_ctas = (CG == 2) ? (int)(gridDim.x >> 1) : (int)gridDim.x;
  const int n_tiles = g.tile_off[g.n_groups];
  const bool snake = g.n_groups > 1;
  const uint32_t base = (smem_u32(dsmem) + 1023u) & ~1023u;
  volatile int* abort_p = &abort_flag;

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&accf_bar[b]), 1);
      mbar_init(smem_u32(&acce_bar[b]), 4 * CG);
    }
    mbar_init(smem_u32(&done_bar), 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    for (int i = 0; i < 3; ++i) {
      prefetch_tmap(&maps.a[i]);
      prefetch_tmap(&maps.b[i]);
    }
  }
  if (warp == 1) {
    tmem_alloc<CG>(smem_u32(&tmem_slot), (uint32_t)p.alloc_cols);
    tmem_relinquish<CG>();
  }
  tc_fence_before();
  if constexpr (CG == 2) cluster_sync(); else __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int qh = 0;
      for (int rd = 0; rd * n_ctas < n_tiles && ok; ++rd) {
        const int t = round_tile(rd, cta, n_ctas, n_tiles, snake);
        if (t < 0) continue;
        Tile T;
        decode_tile<CG, L>(t, p, g, rank, T, qh);
        const CUtensorMap* ma = &maps.a[T.ma];
        const CUtensorMap* mb = &maps.b[T.mb];
        for (int kt = 0; kt < p.Kt; ++kt) {
          if (!mbar_wait(smem_u32(&empty_bar[stage]), phase ^ 1u, p.wd, abort_p, SITE_GEMM_PRODUCER)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&full_bar[stage]);
          uint32_t fbc = fb;
          if constexpr (CG == 1) {
            mbar_arrive_expect_tx(fb, T.tx);
          } else {
            // The leader arms its own full barrier for both CTAs' bytes; the
            // peer only points its TMA completions at that barrier (a
            // completion that lands before the arming leaves the phase pending
            // until the leader's arrival).
            fbc = mapa_shared(fb, 0);
            if (rank == 0) mbar_arrive_expect_tx(fb, 2u * T.tx);
          }
          const uint32_t sbase = base + (uint32_t)stage * p.stage_bytes;
          const uint32_t bbase = sbase + (uint32_t)(L * p.n_atoms) * T.a_part;
#pragma unroll
          for (int h = 0; h < L; ++h) {
            for (int a = 0; a < p.n_atoms; ++a) {
              const int x = kt * p.BK + a * (p.sw / E);
              const uint32_t da = sbase + (uint32_t)(h * p.n_atoms + a) * T.a_part;
              const uint32_t db = bbase + (uint32_t)(h * p.n_atoms + a) * T.b_part;
              if constexpr (CG == 1) {
                tma_load_2d(da, ma, fb, x, T.arow + h * p.lo_row_a);
                tma_load_2d(db, mb, fb, x, T.brow + h * p.lo_row_b);
              } else {
                tma_load_2d_pair(da, ma, fbc, x, T.arow + h * p.lo_row_a);
                tma_load_2d_pair(db, mb, fbc, x, T.brow + h * p.lo_row_b);
              }
            }
          }
          if (++stage == p.stages) { stage = 0; phase ^= 1u; }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------- MMA issuer
    // the whole warp runs the loop in step; lane 0 issues
    if (rank == 0) {
      MmaRing r{full_bar, empty_bar, acce_bar, 0, 0u, lane == 0 ? 1u : 0u};
      bool ok = true;
      int it = 0;
      int qh = 0;
      for (int rd = 0; rd * n_ctas < n_tiles && ok; ++rd) {
        const int t = round_tile(rd, cta, n_ctas, n_tiles, snake);
        if (t < 0) continue;
        Tile T;
        decode_tile<CG, L>(t, p, g, 0, T, qh);
        const int buf = it % p.nbuf;
        const uint32_t use = (uint32_t)(it / p.nbuf);
        // split release: acce_bar[0] / [1] guard row blocks 0 / 1 of the single buffer
        if (!warp_wait(smem_u32(&acce_bar[buf]), (use & 1u) ^ 1u, p.wd, abort_p, SITE_GEMM_MMA)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d0 = tmem_base + (uint32_t)(buf * p.acc_cols);
        // the stage's MMA shape is fixed for the whole tile: dispatch once
        if (p.sw == 128) {
          if (p.n_atoms == 1)
            ok = T.n_mblk == 1 ? mma_tile<CG, KIND, TA, 1, 4, 1>(r, p, T, d0, base, tmem_base, use, abort_p)
                               : mma_tile<CG, KIND, TA, 1, 4, 2>(r, p, T, d0, base, tmem_base, use, abort_p);
          else
            ok = T.n_mblk == 1 ? mma_tile<CG, KIND, TA, 2, 4, 1>(r, p, T, d0, base, tmem_base, use, abort_p)
                               : mma_tile<CG, KIND, TA, 2, 4, 2>(r, p, T, d0, base, tmem_base, use, abort_p);
        } else {
          ok = T.n_mblk == 1 ? mma_tile<CG, KIND, TA, 1, 2, 1>(r, p, T, d0, base, tmem_base, use, abort_p)
                             : mma_tile<CG, KIND, TA, 1, 2, 2>(r, p, T, d0, base, tmem_base, use, abort_p);
        }
        if (!ok) break;
        if constexpr (CG == 1) umma_commit(smem_u32(&accf_bar[buf]), r.issue);
        else umma_commit_pair(smem_u32(&accf_bar[buf]), (uint16_t)3, r.issue);
        ++it;
      }
      // all MMAs of the issuing lane complete before the teardown frees TMEM
      if constexpr (CG == 1) umma_commit(smem_u32(&done_bar), r.issue);
      else umma_commit_pair(smem_u32(&done_bar), (uint16_t)1, r.issue);
      mbar_wait(smem_u32(&done_bar), 0u, p.wd, nullptr, SITE_GEMM_TEARDOWN);
      __syncwarp();
    }
  } else {
    // --------------------------------------------------------------- epilogue
    const int q = warp & 3;                               // TMEM lane quarter of this warp
    float scale = 1.f;
    if constexpr (KIND == 2) scale = 1.f / (__ldg(p.scales) * __ldg(p.scales + 1));
    const bool vec = (p.N & 3) == 0;
    const uint32_t stage_base = base + p.staging_off;     // two 4 KB staging buffers per epilogue warp
    uint32_t sb = 0;
    int it = 0;
    int qh = 0;
    for (int rd = 0; rd * n_ctas < n_tiles; ++rd) {
      const int t = round_tile(rd, cta, n_ctas, n_tiles, snake);
      if (t < 0) continue;
      const int buf = it % p.nbuf;
      const uint32_t use = (uint32_t)(it / p.nbuf);
      ++it;
      if (!mbar_wait(smem_u32(&accf_bar[buf]), use & 1u, p.wd, abort_p, SITE_GEMM_EPILOGUE)) break;
      tc_fence_after();
      Tile T;
      decode_tile<CG, L>(t, p, g, rank, T, qh);
      // rows and columns this warp's TMEM lane quarter holds
      int lrow, qcol0, qcols;
      bool lvalid;
      if (T.layout == 1) {
        lrow = 16 * q + lane; lvalid = lane < 16; qcol0 = 0; qcols = T.BN;
      } else if (T.layout == 2) {
        lrow = 32 * (q & 1) + lane; lvalid = true; qcol0 = (q >> 1) * (T.BN / 2); qcols = T.BN / 2;
      } else {
        lrow = 32 * q + lane; lvalid = true; qcol0 = 0; qcols = T.BN;
      }
      const int ccol0 = T.ccol0 + qcol0;
      for (int m = 0; m < T.n_mblk; ++m) {
        const int row = T.crow0 + m * 128 + lrow;
        const bool rvalid = lvalid && row < T.crow_end;
        float* crow = p.C + (size_t)row * p.N;
        for (int j = 0; j < qcols / 32; ++j) {
          uint32_t r[32];
          const uint32_t taddr =
              tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * p.acc_cols + m * T.BN + 32 * j);
          tmem_ld_32x32b_x32(taddr, r);
          tmem_ld_wait();
          const int col0 = ccol0 + 32 * j;
          // TMA store of the warp's 32 x 32 chunk when its rows are 32
          // consecutive rows inside the problem (layouts 0 and 2)
          const int chunk_row0 = T.crow0 + m * 128 + (lrow - lane);
          if (col0 >= p.N) {
            // the chunk lies past the last column: nothing to write
          } else if (p.tma_store && T.layout != 1 && chunk_row0 + 32 <= T.crow_end) {
            const uint32_t sbuf = stage_base + (uint32_t)((q * 2 + (sb & 1)) * 4096);
            if (lane == 0) bulk_wait_read<1>();          // the buffer's previous store has read it
            __syncwarp();
            const uint32_t rowp = sbuf + (uint32_t)lane * 128u;
#pragma unroll
            for (int v = 0; v < 8; ++v) {
              const uint32_t addr = rowp + (uint32_t)((v ^ (lane & 7)) * 16);
              asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr),
                           "f"(__uint_as_float(r[4 * v + 0]) * scale), "f"(__uint_as_float(r[4 * v + 1]) * scale),
                           "f"(__uint_as_float(r[4 * v + 2]) * scale), "f"(__uint_as_float(r[4 * v + 3]) * scale)
                           : "memory");
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
              tma_store_2d(&maps.c, sbuf, col0, chunk_row0);
              bulk_commit();
            }
            ++sb;
          } else if (rvalid) {
            if (vec && col0 + 32 <= p.N) {
#pragma unroll
              for (int v = 0; v < 8; ++v) {
                float4 o;
                o.x = __uint_as_float(r[4 * v + 0]) * scale;
                o.y = __uint_as_float(r[4 * v + 1]) * scale;
                o.z = __uint_as_float(r[4 * v + 2]) * scale;
                o.w = __uint_as_float(r[4 * v + 3]) * scale;
                *reinterpret_cast<float4*>(crow + col0 + 4 * v) = o;
              }
            } else {
              for (int v = 0; v < 32; ++v)
                if (col0 + v < p.N) crow[col0 + v] = __uint_as_float(r[v]) * scale;
            }
          }
        }
        if (p.split) {
          // this row block is drained: the next tile may start writing it
          tc_fence_before();
          __syncwarp();
          if (lane == 0) {
            const uint32_t eb = smem_u32(&acce_bar[m]);
            if constexpr (CG == 1) mbar_arrive(eb);
            else mbar_arrive_cluster(mapa_shared(eb, 0));
          }
        }
      }
      if (!p.split) {
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          const uint32_t eb = smem_u32(&acce_bar[buf]);
          if constexpr (CG == 1) mbar_arrive(eb);
          else mbar_arrive_cluster(mapa_shared(eb, 0));
        }
      }
    }
    if (lane == 0) bulk_wait_all();                       // staged stores complete before exit
  }

  // ---------------------------------------------------------------- teardown
  tc_fence_before();
  __syncthreads();
  if constexpr (CG == 2) cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc<CG>(tmem_base, (uint32_t)p.alloc_cols);
  }
}

// --------------------------------------------------------------- operand prep
// Row-major FP32 inputs to the tensor-core operand formats.  HBM-bound
// pre-passes outside the GEMM proper.
__device__ __forceinline__ float tf32_rn(float x) {
  // round to nearest even at mantissa bit 13 (finite inputs)
  uint32_t b = __float_as_uint(x);
  if ((b & 0x7f800000u) == 0x7f800000u) return x;
  b = (b + 0xfffu + ((b >> 13) & 1u)) & 0xffffe000u;
  return __uint_as_float(b);
}

__global__ void amax_kernel(const float* __restrict__ x, int64_t n, unsigned int* __restrict__ amax_bits) {
  float m = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(__ldg(x + i)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax_bits, __float_as_uint(m));
}

__device__ __forceinline__ float fp8_scale_of(unsigned int amax_bits) {
  const float amax = __uint_as_float(amax_bits);
  return amax > 0.f ? 448.f / amax : 1.f;
}

// Row-major [R, C] FP32 -> same layout in the operand format (A side).
__global__ void convert_rows_kernel(const float* __restrict__ x, int64_t n, int mode, void* __restrict__ y,
                                    float* __restrict__ y_lo, const unsigned int* __restrict__ amax_bits,
                                    float* __restrict__ scale_out) {
  float s = 1.f;
  if (mode == PM_FP8E4M3) {
    s = fp8_scale_of(*amax_bits);
    if (blockIdx.x == 0 && threadIdx.x == 0 && scale_out) *scale_out = s;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = __ldg(x + i);
    if (mode == PM_BF16) {
      static_cast<__nv_bfloat16*>(y)[i] = __float2bfloat16_rn(v);
    } else if (mode == PM_FP8E4M3) {
      static_cast<__nv_fp8_storage_t*>(y)[i] = __nv_cvt_float_to_fp8(v * s, __NV_SATFINITE, __NV_E4M3);
    } else {
      const float hi = tf32_rn(v);
      static_cast<float*>(y)[i] = hi;
      y_lo[i] = tf32_rn(v - hi);
    }
  }
}

// Row-major [K, N] FP32 -> K-major [N, K] operand (B side), 32x32 tiles.
__global__ void transpose_convert_kernel(const float* __restrict__ x, int K, int N, int mode, void* __restrict__ y,
                                         float* __restrict__ y_lo, const unsigned int* __restrict__ amax_bits,
                                         float* __restrict__ scale_out) {
  __shared__ float tile[32][33];
  float s = 1.f;
  if (mode == PM_FP8E4M3) {
    s = fp8_scale_of(*amax_bits);
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0 && scale_out) *scale_out = s;
  }
  const int n0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, nn = n0 + threadIdx.x;
    tile[r][threadIdx.x] = (k < K && nn < N) ? __ldg(x + (size_t)k * N + nn) : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int nn = n0 + r, k = k0 + threadIdx.x;
    if (nn < N && k < K) {
      const float v = tile[threadIdx.x][r];
      const size_t o = (size_t)nn * K + k;
      if (mode == PM_BF16) {
        static_cast<__nv_bfloat16*>(y)[o] = __float2bfloat16_rn(v);
      } else if (mode == PM_FP8E4M3) {
        static_cast<__nv_fp8_storage_t*>(y)[o] = __nv_cvt_float_to_fp8(v * s, __NV_SATFINITE, __NV_E4M3);
      } else {
        const float hi = tf32_rn(v);
        static_cast<float*>(y)[o] = hi;
        y_lo[o] = tf32_rn(v - hi);
      }
    }
  }
}

// ------------------------------------------------------------------ host side
static inline int dt_elem(int dt) { return dt == PM_FP32 ? 4 : (dt == PM_BF16 ? 2 : 1); }
static inline int dt_halves(int dt) { return dt == PM_FP32 ? 2 : 1; }

bool gemm_tile_valid(int BM, int BN, int BK, int s, int g, int dt, int tmem_a) {
  if (!(BM == 64 || BM == 128 || BM == 256) || !(BN == 64 || BN == 128 || BN == 256)) return false;
  if (dt == PM_FP32) {
    if (BK != 32 && BK != 64) return false;
  } else if (dt == PM_BF16 || dt == PM_FP8E4M3) {
    if (BK != 64 && BK != 128) return false;
  } else {
    return false;
  }
  if (s < 2 || s > kMaxStages || (g != 1 && g != 2)) return false;
  const int64_t stage = (int64_t)dt_halves(dt) * dt_elem(dt) * BK * (BM + BN / g);
  if ((int64_t)s * stage > 232448 - 2048) return false;
  const int n_mblk = (BM + 127) / 128;
  if (n_mblk * BN > 512) return false;
  if (tmem_a == 1) {
    // strategy B: one SM, 128-row blocks, accumulator plus a TMEM copy of
    // every stage's A tile within the 512 columns
    if (g != 1 || BM < 128) return false;
    if (n_mblk * BN + s * n_mblk * dt_halves(dt) * (BK * dt_elem(dt) / 4) > 512) return false;
  } else if (tmem_a != 0) {
    return false;
  }
  return true;
}

struct TmapKey {
  const void* ptr;
  uint64_t rows, cols;
  uint32_t box_rows, box_cols;
  int dt, sw;
  bool operator==(const TmapKey& o) const {
    return ptr == o.ptr && rows == o.rows && cols == o.cols && box_rows == o.box_rows && box_cols == o.box_cols &&
           dt == o.dt && sw == o.sw;
  }
};
struct TmapEntry {
  TmapKey key;
  CUtensorMap map;
  bool used = false;
};
static thread_local TmapEntry g_tmaps[16];
static thread_local int g_tmap_next = 0;

void clear_tmap_caches_this_thread() {
  for (auto& e : g_tmaps) e.used = false;
  g_tmap_next = 0;
  clear_probe_tmap_cache_this_thread();
}

pm_status cached_tmap(CUtensorMap* out, const void* ptr, int dtcode, uint64_t rows, uint64_t cols, uint32_t box_rows,
                      uint32_t box_cols, int sw) {
  TmapKey k{ptr, rows, cols, box_rows, box_cols, dtcode, sw};
  for (auto& e : g_tmaps)
    if (e.used && e.key == k) {
      *out = e.map;
      return PM_OK;
    }
  TmapEntry& e = g_tmaps[g_tmap_next];
  g_tmap_next = (g_tmap_next + 1) % 16;
  pm_status st = make_tmap_2d(&e.map, ptr, dtcode, rows, cols, box_rows, box_cols, sw);
  if (st != PM_OK) {
    e.used = false;
    return st;
  }
  e.key = k;
  e.used = true;
  *out = e.map;
  return PM_OK;
}

template <int CG, int KIND, int TA>
static pm_status launch_gemm(const TensorMaps& maps, const GroupTable& g, const GemmParams& p, int grid,
                             size_t smem, cudaStream_t s) {
  auto kern = gemm_kernel<CG, KIND, TA>;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [&] {
    attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448 - 1024);
  });
  if (attr_err != cudaSuccess) return cuda_fail(attr_err, "cudaFuncSetAttribute(gemm_kernel)");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(kGemmThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (CG == 2) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, maps, g, p);
  if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchKernelEx(gemm_kernel)");
  return PM_OK;
}

static int size_index(int v) { return v == 64 ? 0 : (v == 128 ? 1 : 2); }

// Plans one launch over G problems sharing N, K, BK, stages and cta_group:
// group q is C_q[M_q, N] = A_q B_q with tile BM_q x BN_q.  A_op stacks the A_q
// (rows row0_q ..), B_op stacks the K-major B_q (b_rows_per_group rows each;
// 0 means all groups share one B of N rows).
struct LaunchPlan {
  TensorMaps maps;
  GroupTable g;
  GemmParams p;
  size_t smem = 0;
  int grid = 0;
};

static pm_status plan_launch(int dt, int cg, int BK, int stages, int tmem_a, int G, const int32_t* M, int N, int K,
                             const int16_t* BMv, const int16_t* BNv, bool stacked_b, const void* A_op,
                             const void* B_op, float* C, const float* scales, LaunchPlan& P) {
  PM_REQUIRE(G >= 1 && G <= kMaxGroups, PM_EINVAL, "number of groups %d outside [1, %d]", G, kMaxGroups);
  PM_REQUIRE(N > 0 && K > 0, PM_EINVAL, "N and K must be positive");
  const int e = dt_elem(dt), L = dt_halves(dt);
  PM_REQUIRE(dt >= 0 && dt <= 2, PM_EUNSUPPORTED, "dtype %d is not a pm_dtype", dt);
  int64_t sum_m = 0;
  for (int q = 0; q < G; ++q) {
    PM_REQUIRE(M[q] > 0, PM_EINVAL, "M of group %d must be positive", q);
    PM_REQUIRE(gemm_tile_valid(BMv[q], BNv[q], BK, stages, cg, dt, tmem_a), PM_EUNSUPPORTED,
               "tile configuration BM=%d BN=%d BK=%d stages=%d cta_group=%d dtype=%d tmem_a=%d is outside the "
               "valid space", BMv[q], BNv[q], BK, stages, cg, dt, tmem_a);
    sum_m += M[q];
  }
  PM_REQUIRE(((int64_t)K * e) % 16 == 0, PM_EINVAL, "K*%d bytes must be a multiple of 16", e);
  const int64_t b_rows = stacked_b ? (int64_t)G * N : N;
  PM_REQUIRE(sum_m * L < (1ll << 31) && b_rows * L < (1ll << 31), PM_EINVAL, "too many rows for one launch");
  PM_REQUIRE(A_op && B_op && C, PM_EINVAL, "null operand or output pointer");
  PM_REQUIRE(dt != PM_FP8E4M3 || scales, PM_EINVAL, "FP8 GEMM needs scales_dev");
  GemmParams& p = P.p;
  GroupTable& g = P.g;
  p.N = N;
  p.BK = BK;
  p.stages = stages;
  p.Kt = (K + BK - 1) / BK;
  p.sw = std::min(128, BK * e);
  p.n_atoms = BK * e / p.sw;
  p.ab_fmt = dt == PM_BF16 ? 1u : (dt == PM_FP32 ? 2u : 0u);
  p.lo_row_a = L == 2 ? (int)sum_m : 0;
  p.lo_row_b = L == 2 ? (int)b_rows : 0;
  g.n_groups = G;
  g.tile_off[0] = 0;
  int acc = 0, max_mblk = 1;
  uint32_t stage = 0;
  bool used_m[3] = {false, false, false}, used_n[3] = {false, false, false};
  // rows of each problem in the stacked A and C (the caller's order), then
  // the table's order: largest tile (BM x BN) first, ties in the caller's
  // order (the schedule round_tile describes)
  int64_t row_of[kMaxGroups];
  int order[kMaxGroups];
  for (int64_t q = 0, r0 = 0; q < G; r0 += M[q], ++q) {
    row_of[q] = r0;
    order[q] = (int)q;
  }
  if (G > 1)
    std::stable_sort(order, order + G, [&](int a, int b) { return (int)BMv[a] * BNv[a] > (int)BMv[b] * BNv[b]; });
  for (int i = 0; i < G; ++i) {
    const int q = order[i];
    const int bm = BMv[q], bn = BNv[q];
    g.row0[i] = (int)row_of[q];
    g.rows[i] = M[q];
    g.brow0[i] = stacked_b ? q * N : 0;
    g.tiles_m[i] = (M[q] + cg * bm - 1) / (cg * bm);
    g.tiles_n[i] = (N + bn - 1) / bn;
    const int64_t off = (int64_t)g.tile_off[i] + (int64_t)g.tiles_m[i] * g.tiles_n[i];
    PM_REQUIRE(off < (1ll << 31), PM_EINVAL, "too many tiles");
    g.tile_off[i + 1] = (int)off;
    g.bm_idx[i] = (uint8_t)size_index(bm);
    g.bn_idx[i] = (uint8_t)size_index(bn);
    used_m[g.bm_idx[i]] = used_n[g.bn_idx[i]] = true;
    const int n_mblk = (bm + 127) / 128;
    acc = std::max(acc, (bm < 128 && cg == 2) ? bn / 2 : n_mblk * bn);
    max_mblk = std::max(max_mblk, n_mblk);
    stage = std::max(stage, (uint32_t)(L * p.n_atoms) * (uint32_t)(bm + bn / cg) * (uint32_t)p.sw);
  }
  p.acc_cols = acc;
  // strategy B: one 8-column slot per 128-row x 32-byte A slice, per stage
  p.a_cols = tmem_a ? L * (BK * e / 4) * max_mblk : 0;
  const int a_ring = stages * p.a_cols;
  p.nbuf = (2 * acc + a_ring <= 512) ? 2 : 1;
  // split release when one buffer of two 128-row blocks holds the whole tile
  // (every group: BM = 256 per CTA) and nothing else lives in TMEM
  bool all_two_blocks = true;
  for (int q = 0; q < G; ++q) all_two_blocks = all_two_blocks && BMv[q] == 256;
  p.split = (p.nbuf == 1 && all_two_blocks && tmem_a == 0) ? 1 : 0;
  p.a_col0 = p.nbuf * acc;
  int cols = 32;
  while (cols < p.nbuf * acc + a_ring) cols <<= 1;
  p.alloc_cols = cols;
  p.stage_bytes = stage;
  P.smem = (size_t)stages * stage + 1024;
  // TMA-store epilogue: eight 4 KB staging buffers after the ring, when they fit
  p.staging_off = (uint32_t)stages * stage;
  p.tma_store = 0;
  const bool c_ok = (N % 4) == 0 && ((uintptr_t)C & 15) == 0;
  if (c_ok && P.smem + 32768 <= (size_t)(232448 - 1024)) {
    pm_status st = cached_tmap(&P.maps.c, C, TMAP_F32, (uint64_t)sum_m, (uint64_t)N, 32u, 32u, 128);
    if (st != PM_OK) return st;
    p.tma_store = 1;
    P.smem += 32768;
  }
  const int dtcode = dt == PM_BF16 ? TMAP_BF16 : (dt == PM_FP32 ? TMAP_F32 : TMAP_U8);
  int first_m = -1, first_n = -1;
  for (int i = 0; i < 3; ++i) {
    if (used_m[i]) {
      pm_status st = cached_tmap(&P.maps.a[i], A_op, dtcode, (uint64_t)L * sum_m, (uint64_t)K,
                                 (uint32_t)(64 << i), (uint32_t)(p.sw / e), p.sw);
      if (st != PM_OK) return st;
      if (first_m < 0) first_m = i;
    }
    if (used_n[i]) {
      pm_status st = cached_tmap(&P.maps.b[i], B_op, dtcode, (uint64_t)L * b_rows, (uint64_t)K,
                                 (uint32_t)((64 << i) / cg), (uint32_t)(p.sw / e), p.sw);
      if (st != PM_OK) return st;
      if (first_n < 0) first_n = i;
    }
  }
  for (int i = 0; i < 3; ++i) {          // unused slots hold a valid copy (never dereferenced by a tile)
    if (!used_m[i]) P.maps.a[i] = P.maps.a[first_m];
    if (!used_n[i]) P.maps.b[i] = P.maps.b[first_n];
  }
  unsigned int* w = watchdog_word();
  PM_REQUIRE(w != nullptr, PM_ECUDA, "watchdog word unavailable");
  p.wd = Watchdog{w, watchdog_limit_ns()};
  p.C = C;
  p.scales = scales;
  const int sms = sm_count();
  const int n_tiles = g.tile_off[G];
  P.grid = cg == 1 ? std::min(n_tiles, sms) : 2 * std::min(n_tiles, sms / 2);
  return PM_OK;
}

static pm_status run_plan(const LaunchPlan& P, int dt, int cg, int tmem_a, cudaStream_t s) {
  if (tmem_a) {
    if (dt == PM_BF16) return launch_gemm<1, 0, 1>(P.maps, P.g, P.p, P.grid, P.smem, s);
    if (dt == PM_FP32) return launch_gemm<1, 1, 1>(P.maps, P.g, P.p, P.grid, P.smem, s);
    return launch_gemm<1, 2, 1>(P.maps, P.g, P.p, P.grid, P.smem, s);
  }
  if (cg == 1) {
    if (dt == PM_BF16) return launch_gemm<1, 0, 0>(P.maps, P.g, P.p, P.grid, P.smem, s);
    if (dt == PM_FP32) return launch_gemm<1, 1, 0>(P.maps, P.g, P.p, P.grid, P.smem, s);
    return launch_gemm<1, 2, 0>(P.maps, P.g, P.p, P.grid, P.smem, s);
  }
  if (dt == PM_BF16) return launch_gemm<2, 0, 0>(P.maps, P.g, P.p, P.grid, P.smem, s);
  if (dt == PM_FP32) return launch_gemm<2, 1, 0>(P.maps, P.g, P.p, P.grid, P.smem, s);
  return launch_gemm<2, 2, 0>(P.maps, P.g, P.p, P.grid, P.smem, s);
}

pm_status gemm_launch(const pm_cfg& c, const void* A_op, const void* B_op, float* C, const float* scales,
                      cudaStream_t s) {
  PM_REQUIRE(c.kind == PM_KIND_GEMM, PM_EINVAL, "cfg.kind must be PM_KIND_GEMM");
  PM_REQUIRE(c.M > 0 && c.N > 0 && c.K > 0, PM_EINVAL, "M, N, K must be positive");
  PM_REQUIRE(gemm_tile_valid(c.BM, c.BN, c.BK, c.stages, c.cta_group, c.dtype, c.tmem_a), PM_EUNSUPPORTED,
             "tile configuration BM=%d BN=%d BK=%d stages=%d cta_group=%d dtype=%d tmem_a=%d is outside the "
             "valid space", c.BM, c.BN, c.BK, c.stages, c.cta_group, c.dtype, c.tmem_a);
  static thread_local LaunchPlan P;
  const int32_t M = c.M;
  const int16_t BM = c.BM, BN = c.BN;
  pm_status st = plan_launch(c.dtype, c.cta_group, c.BK, c.stages, c.tmem_a, 1, &M, c.N, c.K, &BM, &BN, false, A_op,
                             B_op, C, scales, P);
  if (st != PM_OK) return st;
  return run_plan(P, c.dtype, c.cta_group, c.tmem_a, s);
}

pm_status grouped_launch(int G, const int32_t* M, int N, int K, const int16_t* BM, const int16_t* BN, int BK,
                         int stages, int cg, const void* A_op, const void* B_op, float* C, cudaStream_t s) {
  static thread_local LaunchPlan P;
  pm_status st = plan_launch(PM_BF16, cg, BK, stages, 0, G, M, N, K, BM, BN, true, A_op, B_op, C, nullptr, P);
  if (st != PM_OK) return st;
  return run_plan(P, PM_BF16, cg, 0, s);
}

}  // namespace pm

using namespace pm;

extern "C" pm_status pm_gemm_operand_bytes(int32_t dtype, int32_t M, int32_t N, int32_t K, size_t* a_bytes,
                                           size_t* b_bytes) {
  PM_REQUIRE(a_bytes && b_bytes, PM_EINVAL, "null output pointer");
  PM_REQUIRE(dtype >= 0 && dtype <= 2 && M > 0 && N > 0 && K > 0, PM_EINVAL, "bad dtype or shape");
  *a_bytes = (size_t)dt_halves(dtype) * dt_elem(dtype) * (size_t)M * K;
  *b_bytes = (size_t)dt_halves(dtype) * dt_elem(dtype) * (size_t)N * K;
  return PM_OK;
}

extern "C" pm_status pm_gemm_prepare(int32_t dtype, const float* A_dev, const float* B_dev, int32_t M, int32_t N,
                                     int32_t K, void* A_op_dev, void* B_op_dev, float* scales_dev, void* stream) {
  PM_REQUIRE(dtype >= 0 && dtype <= 2 && M > 0 && N > 0 && K > 0, PM_EINVAL, "bad dtype or shape");
  PM_REQUIRE(A_dev && B_dev && A_op_dev && B_op_dev, PM_EINVAL, "null pointer");
  PM_REQUIRE(dtype != PM_FP8E4M3 || scales_dev, PM_EINVAL, "FP8 needs scales_dev (4 floats)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int sms = std::max(1, sm_count());
  const int64_t nA = (int64_t)M * K, nB = (int64_t)K * N;
  unsigned int* amax = nullptr;
  if (dtype == PM_FP8E4M3) {
    amax = reinterpret_cast<unsigned int*>(scales_dev + 2);
    PM_CUDA(cudaMemsetAsync(amax, 0, 2 * sizeof(unsigned int), s));
    amax_kernel<<<sms * 4, 256, 0, s>>>(A_dev, nA, amax);
    amax_kernel<<<sms * 4, 256, 0, s>>>(B_dev, nB, amax + 1);
    pm_status st = launch_status("amax_kernel");
    if (st != PM_OK) return st;
  }
  float* a_lo = dtype == PM_FP32 ? static_cast<float*>(A_op_dev) + nA : nullptr;
  float* b_lo = dtype == PM_FP32 ? static_cast<float*>(B_op_dev) + (int64_t)N * K : nullptr;
  convert_rows_kernel<<<sms * 8, 256, 0, s>>>(A_dev, nA, dtype, A_op_dev, a_lo, amax,
                                              dtype == PM_FP8E4M3 ? scales_dev : nullptr);
  pm_status st = launch_status("convert_rows_kernel");
  if (st != PM_OK) return st;
  dim3 grid((N + 31) / 32, (K + 31) / 32);
  PM_REQUIRE(grid.y <= 65535, PM_EINVAL, "K too large for the transpose grid");
  transpose_convert_kernel<<<grid, dim3(32, 8), 0, s>>>(B_dev, K, N, dtype, B_op_dev, b_lo,
                                                          amax ? amax + 1 : nullptr,
                                                          dtype == PM_FP8E4M3 ? scales_dev + 1 : nullptr);
  return launch_status("transpose_convert_kernel");
}

extern "C" pm_status pm_gemm_run(const pm_cfg* cfg, const void* A_op_dev, const void* B_op_dev, float* C_dev,
                                 const float* scales_dev, void* stream) {
  PM_REQUIRE(cfg != nullptr, PM_EINVAL, "cfg is NULL");
  return gemm_launch(*cfg, A_op_dev, B_op_dev, C_dev, scales_dev, static_cast<cudaStream_t>(stream));
}

extern "C" pm_status pm_grouped_gemm_run(int32_t G, const int32_t* M_host, int32_t N, int32_t K,
                                         const int16_t* BM_host, const int16_t* BN_host, int32_t BK,
                                         int32_t stages, int32_t cta_group, const void* A_op_dev,
                                         const void* B_op_dev, float* C_dev, void* stream) {
  PM_REQUIRE(M_host && BM_host && BN_host, PM_EINVAL, "null host array");
  return pm::grouped_launch(G, M_host, N, K, BM_host, BN_host, BK, stages, cta_group, A_op_dev, B_op_dev, C_dev,
                            static_cast<cudaStream_t>(stream));
}

extern "C" pm_status pm_gemm_bench(const pm_cfg* cfg, const void* A_op_dev, const void* B_op_dev, float* C_dev,
                                   const float* scales_dev, int warmup, int reps, void* stream,
                                   pm_probe_result* out) {
  PM_REQUIRE(cfg != nullptr && out != nullptr, PM_EINVAL, "cfg or out is NULL");
  pm::NvtxRange nvtx("pm_gemm_bench");
  PM_REQUIRE(warmup >= 0 && reps >= 1 && reps <= 100000, PM_EINVAL, "warmup >= 0 and 1 <= reps <= 1e5 required");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < warmup; ++i) {
    pm_status st = pm::gemm_launch(*cfg, A_op_dev, B_op_dev, C_dev, scales_dev, s);
    if (st != PM_OK) return st;
  }
  std::vector<cudaEvent_t> ev(2 * (size_t)reps);
  for (auto& e : ev) PM_CUDA(cudaEventCreate(&e));
  pm_status st = PM_OK;
  pm_clock c0, c1;
  pm::read_clock(&c0);
  for (int i = 0; i < reps && st == PM_OK; ++i) {
    cudaEventRecord(ev[2 * i], s);
    st = pm::gemm_launch(*cfg, A_op_dev, B_op_dev, C_dev, scales_dev, s);
    cudaEventRecord(ev[2 * i + 1], s);
  }
  cudaError_t e = cudaStreamSynchronize(s);
  pm::read_clock(&c1);
  std::vector<double> t;
  if (st == PM_OK && e == cudaSuccess)
    for (int i = 0; i < reps; ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
      t.push_back(ms * 1e-3);
    }
  for (auto& x : ev) cudaEventDestroy(x);
  if (st != PM_OK) return st;
  if (e != cudaSuccess) return pm::cuda_fail(e, "cudaStreamSynchronize");
  std::sort(t.begin(), t.end());
  auto q = [&](double f) {
    const double pos = f * (t.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(lo + 1, t.size() - 1);
    return t[lo] + (pos - lo) * (t[hi] - t[lo]);
  };
  out->median_s = q(0.5);
  out->p25_s = q(0.25);
  out->p75_s = q(0.75);
  out->min_s = t.front();
  const double e_b = cfg->dtype == PM_FP32 ? 8.0 : (cfg->dtype == PM_BF16 ? 2.0 : 1.0);
  out->bytes = e_b * ((double)cfg->M * cfg->K + (double)cfg->N * cfg->K) + 4.0 * (double)cfg->M * cfg->N;
  out->final_index = 0;
  pm::clock_record(out, c0, c1);
  unsigned int* w = pm::watchdog_word();
  unsigned int h[2] = {0, 0};
  PM_CUDA(cudaMemcpy(h, w, sizeof(h), cudaMemcpyDeviceToHost));
  if (h[0] != 0) {
    PM_CUDA(cudaMemset(w, 0, 4 * sizeof(unsigned int)));
    pm::set_error("device watchdog expired at site %u", h[1]);
    return PM_ETIMEOUT;
  }
  return PM_OK;
}

extern "C" pm_status pm_gemm_autotune(const pm_cfg* shape, int32_t k, const pm_params* theta_host, int32_t n_sm,
                                      const void* A_op_dev, const void* B_op_dev, float* C_dev,
                                      const float* scales_dev, int warmup, int reps, void* stream,
                                      pm_cfg* pick_out, pm_probe_result* pick_time_out) {
  PM_REQUIRE(shape && theta_host && pick_out, PM_EINVAL, "null argument");
  PM_REQUIRE(k >= 1 && k <= 16, PM_EINVAL, "k must be in [1, 16]");
  pm::NvtxRange nvtx("pm_gemm_autotune");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // model shortlist on the GPU
  char* buf = nullptr;
  const size_t bytes = 16 + (size_t)k * (sizeof(pm_cfg) + sizeof(float));
  PM_CUDA(cudaMallocAsync((void**)&buf, bytes, s));
  int32_t* dmnk = reinterpret_cast<int32_t*>(buf);
  pm_cfg* dpicks = reinterpret_cast<pm_cfg*>(buf + 16);
  float* dt = reinterpret_cast<float*>(buf + 16 + (size_t)k * sizeof(pm_cfg));
  const int32_t mnk[3] = {shape->M, shape->N, shape->K};
  std::vector<pm_cfg> cand(k);
  cudaError_t e = cudaMemcpyAsync(dmnk, mnk, sizeof(mnk), cudaMemcpyHostToDevice, s);
  pm_status st = PM_OK;
  if (e == cudaSuccess) {
    st = pm_autotune_topk(dmnk, 1, shape->dtype, theta_host, n_sm, k, dpicks, dt, stream);
    if (st == PM_OK) e = cudaMemcpyAsync(cand.data(), dpicks, (size_t)k * sizeof(pm_cfg), cudaMemcpyDeviceToHost, s);
  }
  cudaFreeAsync(buf, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (st != PM_OK) return st;
  if (e != cudaSuccess) return pm::cuda_fail(e, "autotune shortlist");
  // time the shortlist with the harness and keep the fastest (first on ties)
  double best = 1e300;
  int bi = -1;
  pm_probe_result best_r = {};
  for (int i = 0; i < k; ++i) {
    if (cand[i].BM == 0) continue;
    pm_probe_result r;
    st = pm_gemm_bench(&cand[i], A_op_dev, B_op_dev, C_dev, scales_dev, warmup, reps, stream, &r);
    if (st != PM_OK) return st;
    if (r.median_s < best) { best = r.median_s; bi = i; best_r = r; }
  }
  PM_REQUIRE(bi >= 0, PM_EUNSUPPORTED, "no valid configuration for this shape");
  *pick_out = cand[bi];
  if (pick_time_out) *pick_time_out = best_r;
  return PM_OK;
}

// ----------------------------------------------------------- host-to-host GEMM
// C_host = A_host B_host with the host link and the GEMM overlapped: B is
// copied and converted first, then A moves in row chunks on a copy stream,
// each chunk is converted and multiplied on a compute stream while the next
// chunk is in flight, and each finished C chunk returns on a third stream.
// Two staging buffers per chunked operand; events order reuse.
namespace pm {

struct HostPipe {
  int dev = -1;
  cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
  cudaEvent_t start, b_ready, done, a_loaded[2], a_free[2], c_ready[2], c_free[2];
};
static thread_local HostPipe g_pipe;

void release_host_pipe_this_thread() {
  HostPipe& P = g_pipe;
  if (P.dev < 0) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cudaSetDevice(P.dev) == cudaSuccess) {
    cudaEvent_t evs[] = {P.start, P.b_ready, P.done, P.a_loaded[0], P.a_loaded[1], P.a_free[0],
                         P.a_free[1], P.c_ready[0], P.c_ready[1], P.c_free[0], P.c_free[1]};
    for (cudaEvent_t e : evs) cudaEventDestroy(e);
    cudaStreamDestroy(P.s_in);
    cudaStreamDestroy(P.s_comp);
    cudaStreamDestroy(P.s_out);
  }
  P = HostPipe();
  if (cur >= 0) cudaSetDevice(cur);
}

static pm_status host_pipe() {
  int dev = 0;
  PM_CUDA(cudaGetDevice(&dev));
  HostPipe& P = g_pipe;
  if (P.dev == dev) return PM_OK;
  PM_REQUIRE(P.dev < 0, PM_EUNSUPPORTED, "pm_gemm_host: one device per host thread");
  PM_CUDA(cudaStreamCreateWithFlags(&P.s_in, cudaStreamNonBlocking));
  PM_CUDA(cudaStreamCreateWithFlags(&P.s_comp, cudaStreamNonBlocking));
  PM_CUDA(cudaStreamCreateWithFlags(&P.s_out, cudaStreamNonBlocking));
  cudaEvent_t* evs[] = {&P.start, &P.b_ready, &P.done, &P.a_loaded[0], &P.a_loaded[1], &P.a_free[0],
                        &P.a_free[1], &P.c_ready[0], &P.c_ready[1], &P.c_free[0], &P.c_free[1]};
  for (cudaEvent_t* e : evs) PM_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  P.dev = dev;
  return PM_OK;
}

struct HostLayout {
  int64_t Mc;
  int chunks;
  size_t off_b32, off_bop, off_a32[2], off_aop[2], off_c[2], off_scales, total;
};

static HostLayout host_layout(const pm_cfg& c, int chunks) {
  HostLayout Lh;
  if (c.dtype == PM_FP8E4M3) chunks = 1;              // the per-tensor scale needs all of A first
  chunks = std::max(1, std::min(chunks, (int)c.M));
  Lh.chunks = chunks;
  Lh.Mc = (c.M + chunks - 1) / chunks;
  const size_t op = (size_t)dt_halves(c.dtype) * dt_elem(c.dtype);
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  size_t o = 0;
  Lh.off_b32 = o; o += up((size_t)c.K * c.N * 4);
  Lh.off_bop = o; o += up(op * c.N * c.K);
  const int nbuf = chunks > 1 ? 2 : 1;
  for (int j = 0; j < 2; ++j) { Lh.off_a32[j] = o; if (j < nbuf) o += up((size_t)Lh.Mc * c.K * 4); }
  for (int j = 0; j < 2; ++j) { Lh.off_aop[j] = o; if (j < nbuf) o += up(op * Lh.Mc * c.K); }
  for (int j = 0; j < 2; ++j) { Lh.off_c[j] = o; if (j < nbuf) o += up((size_t)Lh.Mc * c.N * 4); }
  Lh.off_scales = o; o += 256;
  if (nbuf == 1) {
    Lh.off_a32[1] = Lh.off_a32[0]; Lh.off_aop[1] = Lh.off_aop[0]; Lh.off_c[1] = Lh.off_c[0];
  }
  Lh.total = o;
  return Lh;
}

}  // namespace pm

extern "C" pm_status pm_gemm_host_workspace(const pm_cfg* cfg, int32_t chunks, size_t* bytes) {
  PM_REQUIRE(cfg && bytes, PM_EINVAL, "null argument");
  PM_REQUIRE(cfg->M > 0 && cfg->N > 0 && cfg->K > 0 && cfg->dtype >= 0 && cfg->dtype <= 2, PM_EINVAL,
             "bad shape or dtype");
  *bytes = pm::host_layout(*cfg, chunks).total;
  return PM_OK;
}

extern "C" pm_status pm_gemm_host(const pm_cfg* cfg, const float* A_host, const float* B_host, float* C_host,
                                  void* ws_dev, size_t ws_bytes, int32_t chunks, void* stream) {
  using namespace pm;
  PM_REQUIRE(cfg && A_host && B_host && C_host && ws_dev, PM_EINVAL, "null argument");
  PM_REQUIRE(cfg->kind == PM_KIND_GEMM && cfg->M > 0 && cfg->N > 0 && cfg->K > 0, PM_EINVAL, "bad shape");
  PM_REQUIRE(gemm_tile_valid(cfg->BM, cfg->BN, cfg->BK, cfg->stages, cfg->cta_group, cfg->dtype, cfg->tmem_a),
             PM_EUNSUPPORTED,
             "tile configuration outside the valid space");
  PM_REQUIRE(((uintptr_t)ws_dev & 255) == 0, PM_EINVAL, "workspace must be 256-byte aligned");
  const HostLayout Lh = host_layout(*cfg, chunks);
  PM_REQUIRE(ws_bytes >= Lh.total, PM_ENOMEM, "workspace of %zu bytes is smaller than the %zu needed", ws_bytes,
             Lh.total);
  NvtxRange nvtx("pm_gemm_host");
  pm_status st = host_pipe();
  if (st != PM_OK) return st;
  HostPipe& P = g_pipe;
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(ws_dev);
  const int dt = cfg->dtype;
  const int M = cfg->M, N = cfg->N, K = cfg->K;
  float* b32 = reinterpret_cast<float*>(ws + Lh.off_b32);
  void* bop = ws + Lh.off_bop;
  float* scales = reinterpret_cast<float*>(ws + Lh.off_scales);
  unsigned int* amax = reinterpret_cast<unsigned int*>(scales + 2);
  const int sms = std::max(1, sm_count());
  PM_CUDA(cudaEventRecord(P.start, caller));
  PM_CUDA(cudaStreamWaitEvent(P.s_in, P.start, 0));
  PM_CUDA(cudaStreamWaitEvent(P.s_comp, P.start, 0));
  PM_CUDA(cudaStreamWaitEvent(P.s_out, P.start, 0));
  // B: copy, then convert to the K-major operand
  PM_CUDA(cudaMemcpyAsync(b32, B_host, (size_t)K * N * 4, cudaMemcpyHostToDevice, P.s_in));
  PM_CUDA(cudaEventRecord(P.b_ready, P.s_in));
  PM_CUDA(cudaStreamWaitEvent(P.s_comp, P.b_ready, 0));
  if (dt == PM_FP8E4M3) {
    PM_CUDA(cudaMemsetAsync(amax, 0, 2 * sizeof(unsigned int), P.s_comp));
    amax_kernel<<<sms * 4, 256, 0, P.s_comp>>>(b32, (int64_t)K * N, amax + 1);
  }
  dim3 tgrid((N + 31) / 32, (K + 31) / 32);
  PM_REQUIRE(tgrid.y <= 65535, PM_EINVAL, "K too large for the transpose grid");
  transpose_convert_kernel<<<tgrid, dim3(32, 8), 0, P.s_comp>>>(
      b32, K, N, dt, bop, dt == PM_FP32 ? static_cast<float*>(bop) + (int64_t)N * K : nullptr,
      dt == PM_FP8E4M3 ? amax + 1 : nullptr, dt == PM_FP8E4M3 ? scales + 1 : nullptr);
  st = launch_status("transpose_convert_kernel");
  if (st != PM_OK) return st;
  // A in row chunks
  const int nch = (int)((M + Lh.Mc - 1) / Lh.Mc);
  for (int i = 0; i < nch; ++i) {
    const int j = i & 1;
    const int64_t r0 = (int64_t)i * Lh.Mc;
    const int rows = (int)std::min<int64_t>(Lh.Mc, M - r0);
    float* a32 = reinterpret_cast<float*>(ws + Lh.off_a32[j]);
    void* aop = ws + Lh.off_aop[j];
    float* cd = reinterpret_cast<float*>(ws + Lh.off_c[j]);
    if (i >= 2) PM_CUDA(cudaStreamWaitEvent(P.s_in, P.a_free[j], 0));
    PM_CUDA(cudaMemcpyAsync(a32, A_host + r0 * K, (size_t)rows * K * 4, cudaMemcpyHostToDevice, P.s_in));
    PM_CUDA(cudaEventRecord(P.a_loaded[j], P.s_in));
    PM_CUDA(cudaStreamWaitEvent(P.s_comp, P.a_loaded[j], 0));
    const int64_t nA = (int64_t)rows * K;
    if (dt == PM_FP8E4M3) amax_kernel<<<sms * 4, 256, 0, P.s_comp>>>(a32, nA, amax);
    convert_rows_kernel<<<sms * 8, 256, 0, P.s_comp>>>(a32, nA, dt, aop,
                                                       dt == PM_FP32 ? static_cast<float*>(aop) + nA : nullptr,
                                                       dt == PM_FP8E4M3 ? amax : nullptr,
                                                       dt == PM_FP8E4M3 ? scales : nullptr);
    st = launch_status("convert_rows_kernel");
    if (st != PM_OK) return st;
    PM_CUDA(cudaEventRecord(P.a_free[j], P.s_comp));
    if (i >= 2) PM_CUDA(cudaStreamWaitEvent(P.s_comp, P.c_free[j], 0));
    pm_cfg cc = *cfg;
    cc.M = rows;
    st = gemm_launch(cc, aop, bop, cd, scales, P.s_comp);
    if (st != PM_OK) return st;
    PM_CUDA(cudaEventRecord(P.c_ready[j], P.s_comp));
    PM_CUDA(cudaStreamWaitEvent(P.s_out, P.c_ready[j], 0));
    PM_CUDA(cudaMemcpyAsync(C_host + r0 * N, cd, (size_t)rows * N * 4, cudaMemcpyDeviceToHost, P.s_out));
    PM_CUDA(cudaEventRecord(P.c_free[j], P.s_out));
  }
  PM_CUDA(cudaEventRecord(P.done, P.s_out));
  PM_CUDA(cudaStreamWaitEvent(caller, P.done, 0));
  return PM_OK;
}
