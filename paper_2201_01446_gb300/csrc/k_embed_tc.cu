// Tabulated embedding fused with the environment-matrix contraction on the
// tensor cores (Sec. 3.2-3.4, Eq. 1-2).
//
// Per atom i the contraction regroups by table interval k (exact in real
// arithmetic):
//   T_i[c][m] = (1/N_m) sum_k sum_q C_ik[c][q] c_k[q][m],
//   C_ik[c][q] = sum_{j in interval k} R_ij[c] u_ij^q,
// a dense product of an A matrix with rows (atom, c) and K = (interval, q)
// (q padded from 6 to 8) and the table read as B with N = m.  A CTA owns a
// tile of 32 atoms of one centre type = 128 A rows.  Phase 1 (all warps, one
// warp per atom): pair geometry, counting sort of the pairs by interval
// (deterministic), the sorted (R, u) written to the CTA's scratch (L2
// resident).  Phase 2: the K range is the tile's occupied interval range;
// warp 0 streams the table blocks (2 intervals x M columns, all pieces) with
// bulk async copies, warps 4-7 form C for the same two intervals in the
// stage's A slot (one thread per row), warp 1 issues the MMAs.  Epilogue:
// TMEM -> T (scaled by 1/N_m).  The kernel is persistent (two CTAs per SM),
// so the per-CTA scratch stays small.  Operands are FP32-accurate: each value
// is h + m + l in BF16 and six piece products accumulate in FP32 (the h*h sum
// and the small products in separate TMEM accumulators).
#include <atomic>
#include <cuda_bf16.h>
#include <limits.h>
#include <math.h>

#include "dp_internal.h"
#include "embed_common.cuh"
#include "tc_common.cuh"

namespace {
using namespace dp_embed;
using namespace dp_tc;

constexpr int kPC = 3;            // BF16 pieces per value
constexpr int kNPROD = 6;         // piece products per K step
constexpr int kAtoms = 32;        // atoms per tile
constexpr int kRows = 128;        // A rows per tile (atom, c)
constexpr int kThreads = 256;
constexpr int kNS = 3;            // pipeline stages
constexpr int kABytes = kRows * 16 * 2;  // one piece of an A stage (K = 16)
constexpr int kAcc1 = 128;        // TMEM column of the small-product accumulator
constexpr int kTmemCols = 256;

__host__ __device__ inline int round16(int v) { return (v + 15) & ~15; }
__host__ __device__ inline int even_bins(int nbins) { return (nbins + 1) & ~1; }

// forward table operand, per centre type: K chunk kc = intervals 2kc, 2kc+1;
// its block holds the pieces of the NP x 16 tile, NP = M rounded up to 16
__host__ __device__ inline int64_t tabF_elems(int nbins, int NP) {
  return (int64_t)even_bins(nbins) / 2 * kPC * NP * 16;
}
// backward table operand: N = (interval, q) rows, K = m; per 16-wide m chunk
// kc and piece p one block of all NB8 = 8 * nbins rows
__host__ __device__ inline int64_t tabB_elems(int nbins, int NP) {
  return (int64_t)(NP / 16) * kPC * 8 * even_bins(nbins) * 16;
}

// value of the padded table entry (interval b of centre type ti, power q,
// column m): the normalised quintic coefficient, zero for q >= 6 or m >= M
__device__ __forceinline__ float tab_value(const float* table, int ti, int nbins, int M, int b,
                                           int q, int m) {
  if (b >= nbins || q >= 6 || m >= M) return 0.0f;
  return table[((size_t)ti * nbins + b) * 6 * M + (size_t)q * M + m];
}

__device__ __forceinline__ void split3(float x, __nv_bfloat16& h, __nv_bfloat16& m,
                                       __nv_bfloat16& l) {
  h = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

// forward operand: element (n = m, k = 8 b + q)
__global__ void k_tile_tabF(const float* __restrict__ table, int ntypes, int nbins, int M, int NP,
                            __nv_bfloat16* __restrict__ out) {
  const int nb2 = even_bins(nbins);
  const int64_t per = tabF_elems(nbins, NP) / kPC;  // values per type
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= per * ntypes) return;
  const int ti = (int)(i / per);
  const int64_t r = i - (int64_t)ti * per;
  const int m = (int)(r % NP);
  const int k = (int)(r / NP);  // 0 .. 8 * nb2
  const int b = k >> 3, q = k & 7;
  if (b >= nb2) return;
  __nv_bfloat16 h, md, l;
  split3(tab_value(table, ti, nbins, M, b, q, m), h, md, l);
  const int kc = k >> 4;
  const size_t o = (size_t)ti * tabF_elems(nbins, NP) + (size_t)kc * kPC * NP * 16 + tile_off(m, k & 15);
  out[o] = h;
  out[o + NP * 16] = md;
  out[o + 2 * NP * 16] = l;
}

// backward operand: element (n = 8 b + q, k = m)
__global__ void k_tile_tabB(const float* __restrict__ table, int ntypes, int nbins, int M, int NP,
                            __nv_bfloat16* __restrict__ out) {
  const int NB8 = 8 * even_bins(nbins);
  const int64_t per = (int64_t)NB8 * NP;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= per * ntypes) return;
  const int ti = (int)(i / per);
  const int64_t r = i - (int64_t)ti * per;
  const int n = (int)(r / NP), m = (int)(r % NP);
  __nv_bfloat16 h, md, l;
  split3(tab_value(table, ti, nbins, M, n >> 3, n & 7, m), h, md, l);
  const int kc = m >> 4;
  const size_t blk = (size_t)NB8 * 16;
  const size_t o = (size_t)ti * tabB_elems(nbins, NP) + (size_t)kc * kPC * blk + tile_off(n, m & 15);
  out[o] = h;
  out[o + blk] = md;
  out[o + 2 * blk] = l;
}

struct FwdCfg {
  int NP;         // M rounded up to 16: MMA N
  int bstage;     // bytes of the B part of a stage (all pieces)
  int stage;      // bytes per stage
  int nbp;        // bin ends per atom (uint16, rounded to 8)
  size_t region;  // the stages, or phase 1's per-warp scratch (the larger)
  size_t smem;    // dynamic shared memory
};

// N_m + 32 rounded to 32: the most pairs within rc an atom may have
__host__ __device__ inline int scap_of(const EnvParams& ep) {
  return ((int)(1.0f / ep.inv_nm + 0.5f) + 32 + 31) / 32 * 32;
}

// phase 1's per-warp scratch (int histogram, then the staged pairs: 32 bytes
// each) lives in the stage memory, idle between the previous tile's epilogue
// and this tile's MMAs
__host__ __device__ inline size_t warp_scratch_bytes(const EnvParams& ep) {
  return (size_t)round4(ep.ntypes * ep.n_int) * 4 + (size_t)scap_of(ep) * 32;
}

__host__ __device__ inline FwdCfg fwd_cfg(const EnvParams& ep) {
  FwdCfg c;
  c.NP = round16(ep.M);
  c.bstage = kPC * c.NP * 32;
  c.stage = kPC * kABytes + c.bstage;
  c.nbp = (ep.ntypes * ep.n_int + 7) & ~7;
  c.region = (size_t)kNS * c.stage;
  const size_t p1 = (size_t)(kThreads / 32) * warp_scratch_bytes(ep);
  if (c.region < p1) c.region = p1;
  c.smem = 128 + c.region + (size_t)kAtoms * c.nbp * 2;
  return c;
}

__device__ __forceinline__ int bin_begin16(const uint16_t* hist, int b) {
  return b ? hist[b - 1] : 0;
}

// A tile's occupied units (chunks of two bins, or windows of bins) as a
// bitmask: the first set bit at or after c, or n when there is none.
constexpr int kMaxOccWords = 64;  // 2048 units
__device__ __forceinline__ int next_occ(const uint32_t* occ, int c, int n) {
  for (int w = c >> 5; w * 32 < n; ++w) {
    const uint32_t m = occ[w] & (w == (c >> 5) ? (0xffffffffu << (c & 31)) : 0xffffffffu);
    if (m) {
      const int k = w * 32 + __ffs(m) - 1;
      return k < n ? k : n;
    }
  }
  return n;
}

// bit u of occ: does any atom of the tile have a pair in bins [b0, b1) (of
// the bin ends in shist)?  Units u = 0 .. n - 1 start at bin bs + width * u.
__device__ __forceinline__ void mark_occupied(const uint16_t* shist, int nbp, int nbins, int bs,
                                              int width, int n, uint32_t* occ, int warp,
                                              int lane, int nwarps) {
  for (int w = warp; w * 32 < n; w += nwarps) {
    const int u = w * 32 + lane;
    bool any = false;
    if (u < n) {
      const int b0 = min(bs + width * u, nbins), b1 = min(b0 + width, nbins);
      for (int al = 0; al < kAtoms && !any && b1 > b0; ++al) {
        const uint16_t* hist = shist + al * nbp;
        any = hist[b1 - 1] > bin_begin16(hist, b0);
      }
    }
    const uint32_t m = __ballot_sync(0xffffffffu, any);
    if (lane == 0) occ[w] = m;
  }
}

__device__ __forceinline__ int tile_type(const TileMap& tm, int64_t tile) {
  int ti = 0;
  while (ti + 1 < tm.ntypes && tile >= tm.tile_off[ti + 1]) ++ti;
  return ti;
}

__device__ __forceinline__ int tile_atom(const TileMap& tm, int ti, int64_t tile, int al) {
  const int64_t pos = (tile - tm.tile_off[ti]) * kAtoms + al;
  if (pos >= tm.atom_cnt[ti]) return -1;
  return tm.idx ? tm.idx[tm.atom_off[ti] + pos] : (int)(tm.atom_off[ti] + pos);
}

// Phase 1 for one atom (one warp): one pass over the neighbor list computes
// the geometry of every pair, the histogram of the pairs within rc by bin =
// (neighbor type, interval) and a staged copy of those pairs in list order in
// the warp's shared memory (bin, j, s, u, dx, dy, dz, 1/r); after the
// exclusive scan a second pass over the staged pairs only scatters (R, u) in
// stable bin order into the scratch rows of tile slot al, and (dx, dy, dz, j)
// for the backward.  On return hist holds the end
// of every bin (all zero when the atom has no slot: padding or overflow).
// Returns the pairs within rc; lo/hi the occupied bin range of this atom.
// off: the offsets of the atom's system, whose first atom is jb (neighbor
// entries hold system-local indices; the pair copy gets global ones)
__device__ __forceinline__ int sort_atom(int atom, int jb, const float4* __restrict__ off,
                                         const uint32_t* __restrict__ nlist,
                                         const int32_t* __restrict__ nn, int cap,
                                         const CellGeom& g, const EnvParams& ep, int scap, int* hist,
                                         int nbins, float4* __restrict__ scR,
                                         float* __restrict__ scU, float4* stg,
                                         float4* __restrict__ pout, int lane, int& nrange,
                                         int& nover, int& lo, int& hi) {
  for (int b = lane; b < nbins; b += 32) hist[b] = 0;
  __syncwarp();
  lo = INT_MAX;
  hi = -1;
  if (atom < 0) return 0;
  const float4 oi = off[atom - jb];
  const int cnt = min(nn[atom], cap);
  const uint32_t* L = nlist + (size_t)atom * cap;
  const unsigned below = (1u << lane) - 1u;
  int np = 0;
  // four-deep software pipeline over the list: while round r computes, the
  // offsets of rounds r + 1 .. r + 3 and the list entries of round r + 4 are
  // in flight
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  uint32_t e_cur = lane < cnt ? L[lane] : 0u;
  uint32_t e_n1 = 32 + lane < cnt ? L[32 + lane] : 0u;
  uint32_t e_n2 = 64 + lane < cnt ? L[64 + lane] : 0u;
  uint32_t e_n3 = 96 + lane < cnt ? L[96 + lane] : 0u;
  float4 o_cur = lane < cnt ? off[e_cur >> 5] : z4;
  float4 o_n1 = 32 + lane < cnt ? off[e_n1 >> 5] : z4;
  float4 o_n2 = 64 + lane < cnt ? off[e_n2 >> 5] : z4;
  for (int b0 = 0; b0 < cnt; b0 += 32) {
    const int k = b0 + lane;
    const uint32_t e = e_cur;
    const float4 oj = o_cur;
    o_cur = o_n1;
    o_n1 = o_n2;
    if (k + 96 < cnt) o_n2 = off[e_n3 >> 5];
    e_cur = e_n1;
    e_n1 = e_n2;
    e_n2 = e_n3;
    if (k + 128 < cnt) e_n3 = L[k + 128];
    bool in = false;
    int bin = 0;
    Pair Pk;
    if (k < cnt) {
      float dx, dy, dz;
      int tj;
      pair_from(oi, oj, g, e, dx, dy, dz, tj);
      const float r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < ep.rc2) {
        Pair& P = Pk;
        pair_geom(ep, dx, dy, dz, r2, tj, P);
        bin = tj * ep.n_int + P.th;
        atomicAdd(&hist[bin], 1);
        nrange += P.out_of_range;
        lo = min(lo, bin);
        hi = max(hi, bin);
        in = true;
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, in);
    const int q = np + __popc(bal & below);
    if (in && q < scap) {
      stg[2 * q] = make_float4(__int_as_float(bin), __int_as_float(jb + (int)(e >> 5)), Pk.s, Pk.u);
      stg[2 * q + 1] = make_float4(Pk.dx, Pk.dy, Pk.dz, Pk.ir);
    }
    np += __popc(bal);
  }
  __syncwarp();
  if (np > scap) {
    // more pairs within rc than N_m + 32: an overflow of sel, T_i = 0
    for (int b = lane; b < nbins; b += 32) hist[b] = 0;
    __syncwarp();
    if (lane == 0) ++nover;
    lo = INT_MAX;
    hi = -1;
    return np;
  }
  warp_exclusive_scan(hist, nbins, lane);
  for (int b0 = 0; b0 < np; b0 += 32) {
    const int kk = b0 + lane;
    const bool in = kk < np;
    float4 sa = make_float4(0.f, 0.f, 0.f, 0.f), sb = sa;
    if (in) {
      sa = stg[2 * kk];
      sb = stg[2 * kk + 1];
    }
    const int bin = __float_as_int(sa.x);
    Pair P;
    P.s = sa.z;
    P.u = sa.w;
    P.dx = sb.x;
    P.dy = sb.y;
    P.dz = sb.z;
    P.ir = sb.w;
    const int pos = sorted_slot(hist, in, bin, lane);
    if (in) {
      // the backward's copy: displacement and neighbor index in sorted order
      // (streaming stores, evict-first in L2: read back only by the backward,
      // they should not push the L2-resident scratch out)
      __stcs(pout + pos, make_float4(P.dx, P.dy, P.dz, sa.y));
      // the pair's row of R (one 16-byte record: the four generator threads
      // of the atom read it as one sector) and its u
      scR[pos] = make_float4(P.s, P.s * P.dx * P.ir, P.s * P.dy * P.ir, P.s * P.dz * P.ir);
      scU[pos] = P.u;
    }
  }
  __syncwarp();
  return np;
}

// COMPACT: contract only the occupied chunks of a tile's range (several
// neighbor types); otherwise every chunk of the range
template <bool COMPACT>
__global__ void __launch_bounds__(kThreads, 2)
    k_tab_fwd_tc(int64_t ntile, TileMap tm, const float4* __restrict__ off,
                 const uint32_t* __restrict__ nlist, const int32_t* __restrict__ nn, int cap,
                 CellGeom g, EnvParams ep, const __nv_bfloat16* __restrict__ tabF, int scap,
                 float* __restrict__ scratch, float4* __restrict__ pairs_out,
                 uint16_t* __restrict__ hist_out, int2* __restrict__ range_out,
                 float* __restrict__ T,
                 int32_t* __restrict__ status, unsigned long long* __restrict__ pair_count,
                 const int32_t* __restrict__ sys_of, const int32_t* __restrict__ sys_base,
                 const float4* __restrict__ sys_edge, long long gen_wait_limit) {
  const FwdCfg cf = fwd_cfg(ep);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  uint16_t* shist = (uint16_t*)(base + cf.region);  // [32 atoms][nbp] bin ends
  int* whist = (int*)(base + (size_t)(threadIdx.x >> 5) * warp_scratch_bytes(ep));
  float4* wstg = (float4*)(whist + round4(ep.ntypes * ep.n_int));
  __shared__ __align__(8) uint64_t s_full[kNS], s_empty[kNS], s_gen[kNS], s_acc;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort, s_lo, s_hi;
  __shared__ int s_atom[kAtoms];
  __shared__ uint32_t s_occ[kMaxOccWords];  // occupied chunks of the tile's range
  volatile int* abort_flag = &s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nbins = ep.ntypes * ep.n_int;
  const int M = ep.M, NP = cf.NP;
  const uint32_t b_piece = (uint32_t)NP * 32;
  const int64_t tabF_ti = tabF_elems(nbins, NP);
  float* sc_cta = scratch + (size_t)blockIdx.x * 5 * kAtoms * scap;

  if (tid == 0) {
    for (int s = 0; s < kNS; ++s) {
      mbar_init(&s_full[s], 1);
      mbar_init(&s_empty[s], 1);
      mbar_init(&s_gen[s], kRows);
    }
    mbar_init(&s_acc, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = s_tmem;

  int nrange = 0, nover = 0;
  unsigned long long npairs = 0;
  uint32_t it = 0;     // chunks this CTA has pipelined (the same count in every role)
  uint32_t acc_n = 0;  // accumulator completions
  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int ti = tile_type(tm, tile);
    if (tid == 0) {
      s_lo = INT_MAX;
      s_hi = -1;
    }
    // the stage memory turns from the async proxy's (copies, MMAs) to phase 1's
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    // ---- phase 1: four atoms per warp
    for (int j = 0; j < kAtoms / 8; ++j) {
      const int al = warp * (kAtoms / 8) + j;
      const int atom = tile_atom(tm, ti, tile, al);
      if (lane == 0) s_atom[al] = atom;
      int lo, hi;
      // several systems in one launch: the atom's system gives the base of
      // its offsets and the cell edges of the stencil shifts
      int jb = 0;
      CellGeom gs = g;
      if (sys_of && atom >= 0) {
        const int sy = sys_of[atom];
        jb = sys_base[sy];
        const float4 e4 = sys_edge[sy];
        gs.edgef[0] = e4.x;
        gs.edgef[1] = e4.y;
        gs.edgef[2] = e4.z;
      }
      const int np = sort_atom(atom, jb, off + jb, nlist, nn, cap, gs, ep, scap, whist, nbins,
                               reinterpret_cast<float4*>(sc_cta) + (size_t)al * scap,
                               sc_cta + 4 * (size_t)kAtoms * scap + (size_t)al * scap, wstg,
                               pairs_out + ((size_t)tile * kAtoms + al) * scap, lane, nrange,
                               nover, lo, hi);
      // bin ends of this atom (<= N_m + 32 < 2^16)
      for (int b = lane; b < cf.nbp; b += 32)
        shist[al * cf.nbp + b] = (uint16_t)(b < nbins ? whist[b] : 0);
      npairs += (unsigned long long)np;
      lo = __reduce_min_sync(0xffffffffu, lo);
      hi = __reduce_max_sync(0xffffffffu, hi);
      if (lane == 0 && hi >= 0) {
        atomicMin(&s_lo, lo);
        atomicMax(&s_hi, hi);
      }
    }
    // the stage memory goes back to the async proxy (this tile's copies)
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    const int kb0 = s_hi >= 0 ? (s_lo & ~1) : 0;
    const int nk = s_hi >= 0 ? (s_hi - kb0) / 2 + 1 : 0;  // chunks of two bins
    // the backward's copy of the tile's bin ends and occupied range
    {
      int4* ho = reinterpret_cast<int4*>(hist_out + (size_t)tile * kAtoms * cf.nbp);
      const int4* hs = reinterpret_cast<const int4*>(shist);
      for (int q = tid; q < kAtoms * cf.nbp / 8; q += kThreads) __stcs(ho + q, hs[q]);
      if (tid == 0) range_out[tile] = make_int2(kb0, nk);
    }
    // the chunks of the range with a pair (bit kc of s_occ): with several
    // neighbor types the range spans every type's section of the bins and
    // much of it is empty, and the contraction skips those chunks (every role
    // walks the same list).  With one neighbor type the occupied bins form
    // one thermally broadened band; there the pass costs more than it saves
    // (measured on 4M-atom copper) and every chunk of the range is taken.
    int nocc = nk;
    if (COMPACT) {
      mark_occupied(shist, cf.nbp, nbins, kb0, 2, nk, s_occ, warp, lane, kThreads / 32);
      __syncthreads();
      nocc = 0;  // popcount of the mask over [0, nk)
      for (int w = 0; w * 32 < nk; ++w)
        nocc += __popc(s_occ[w] & (nk - w * 32 >= 32 ? 0xffffffffu : (1u << (nk - w * 32)) - 1u));
    }
    auto next_kc = [&](int kc) { return COMPACT ? next_occ(s_occ, kc, nk) : kc; };
    // ---- phase 2: T rows of the tile = C . table over the occupied bins
    if (nk > 0) {
      if (warp == 0) {
        if (lane == 0) {
          const __nv_bfloat16* Bt = tabF + (size_t)ti * tabF_ti + (size_t)(kb0 / 2) * kPC * NP * 16;
          uint32_t i = it;
          int kc = next_kc(0);
          for (; kc < nk; kc = next_kc(kc + 1), ++i) {
            const int s = i % kNS;
            const uint32_t u = i / kNS;
            if (u > 0 && !mbar_wait(&s_empty[s], (u - 1) & 1, abort_flag)) break;
            mbar_expect_tx(&s_full[s], kPC * b_piece);
            bulk_g2s(smem_u32(base + (size_t)s * cf.stage + kPC * kABytes),
                     Bt + (size_t)kc * kPC * NP * 16, kPC * b_piece, &s_full[s]);
          }
          if (kc < nk) {
            // aborted: wait (bounded) for the copies already issued to land
            for (uint32_t j = (i - it) > (uint32_t)kNS ? i - kNS : it; j < i; ++j)
              mbar_wait(&s_full[j % kNS], (j / kNS) & 1, nullptr);
          }
        }
        __syncwarp();
      } else if (warp == 1) {
        if (lane == 0) {
          const uint32_t idesc = make_idesc_bf16(kRows, NP);
          uint32_t i = it;
          for (int kc = 0; kc < nocc; ++kc, ++i) {  // kc: the index among the occupied
            const int s = i % kNS;
            const uint32_t u = i / kNS;
            if (!mbar_wait(&s_full[s], u & 1, abort_flag)) break;
            if (!mbar_wait(&s_gen[s], u & 1, abort_flag)) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            const uint32_t st0 = smem_u32(base + (size_t)s * cf.stage);
#pragma unroll
            for (int q = 0; q < kNPROD; ++q) {
              int pa, pb;
              prod_pieces(q, pa, pb);
              const uint64_t ad = make_desc(st0 + pa * kABytes, 128, 256);
              const uint64_t bd = make_desc(st0 + kPC * kABytes + pb * b_piece, 128, 256);
              const uint32_t dst = tmem + (q > 0 ? (uint32_t)kAcc1 : 0u);
              const uint32_t acc = (kc > 0 || q > 1) ? 1u : 0u;
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dst),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    smem_u32(&s_empty[s])));
          }
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                  smem_u32(&s_acc)));
        }
        __syncwarp();
      } else if (warp >= 4) {
        // C rows: thread r = (atom al, component c), two bins per chunk.  The
        // pairs of the tile's chunks are one contiguous sorted range per atom,
        // read in groups of four; the next group (of this chunk or the next)
        // is always in flight while the current one is computed
        const int r = tid - 128, al = r >> 2, c = r & 3;
        const uint16_t* hist = shist + al * cf.nbp;
        const size_t st = (size_t)kAtoms * scap;
        const float* Rc = sc_cta + (size_t)al * scap * 4 + c;  // stride 4: R records
        const float* Us = sc_cta + 4 * st + (size_t)al * scap;
        auto bounds = [&](int kc, int& kb, int& km, int& ke) {
          const int b0 = kb0 + 2 * kc;
          kb = bin_begin16(hist, min(b0, nbins));
          km = b0 < nbins ? hist[b0] : kb;
          ke = b0 + 1 < nbins ? hist[b0 + 1] : km;
        };
        float rv[4], uv[4];
        auto load4 = [&](int k, int ke) {
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const bool ok = k + t < ke;
            rv[t] = ok ? Rc[4 * (k + t)] : 0.0f;
            uv[t] = ok ? Us[k + t] : 0.0f;
          }
        };
        int kbeg, kmid, kend;
        int kc = next_kc(0);
        bounds(kc, kbeg, kmid, kend);
        load4(kbeg, kend);
        uint32_t i = it;
        for (; kc < nk; ++i) {
          const int s = i % kNS;
          const uint32_t u = i / kNS;
          const int kn = next_kc(kc + 1);
          int nbeg = 0, nmid = 0, nend = 0;
          if (kn < nk) bounds(kn, nbeg, nmid, nend);
          float x[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) x[q] = 0.0f;
          if (kbeg >= kend) load4(nbeg, nend);  // empty chunk: on to the next
          for (int k = kbeg; k < kend; k += 4) {
            float cr[4], cu[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              cr[t] = rv[t];
              cu[t] = uv[t];
            }
            if (k + 4 < kend) load4(k + 4, kend);
            else load4(nbeg, nend);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const float uu = cu[t], u2 = uu * uu;
              const float ra = k + t < kmid ? cr[t] : 0.0f;  // first bin
              const float rb = cr[t] - ra;                   // second bin (or padding 0)
              const float pw[6] = {1.0f, uu, u2, u2 * uu, u2 * u2, u2 * u2 * uu};
#pragma unroll
              for (int q = 0; q < 6; ++q) {
                x[q] = fmaf(ra, pw[q], x[q]);
                x[8 + q] = fmaf(rb, pw[q], x[8 + q]);
              }
            }
          }
          kbeg = nbeg;
          kmid = nmid;
          kend = nend;
          kc = kn;
          // (gen_wait_limit: the full limit; a test shortens this one wait,
          // on the MMAs' release of the stage, to make it run out: every wait
          // that drains the CTA's own copies and MMAs keeps the full limit)
          if (u > 0 && !mbar_wait_lim(&s_empty[s], (u - 1) & 1, abort_flag, gen_wait_limit))
            break;
          unsigned char* sa = base + (size_t)s * cf.stage;
#pragma unroll
          for (int hb = 0; hb < 2; ++hb) {
            __align__(16) __nv_bfloat16 pv[3][8];
            split8<kPC>(x + 8 * hb, pv);
            const int o = (r >> 3) * 256 + hb * 128 + (r & 7) * 16;
#pragma unroll
            for (int p = 0; p < kPC; ++p)
              *reinterpret_cast<uint4*>(sa + p * kABytes + o) = *reinterpret_cast<const uint4*>(pv[p]);
          }
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
          mbar_arrive(&s_gen[s]);
        }
      }
      it += nocc;
      if (!mbar_wait(&s_acc, acc_n & 1, nullptr)) *abort_flag = 1;
      ++acc_n;
      asm volatile("tcgen05.fence::after_thread_sync;\n");
    }
    __syncthreads();
    if (*abort_flag) break;
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4).. and half the columns
    {
      const int lg = warp & 3, half = warp >> 2;
      const int row_t = lg * 32 + lane;
      const int al = row_t >> 2, c = row_t & 3;
      const int atom = s_atom[al];
      const uint32_t tbase = tmem + ((uint32_t)(lg * 32) << 16);
      const int nch = NP / 16;
      const int c_beg = half ? (nch + 1) / 2 : 0, c_end = half ? nch : (nch + 1) / 2;
      float* Tr = atom >= 0 ? T + (size_t)atom * 4 * M + (size_t)c * M : nullptr;
      for (int ch = c_beg; ch < c_end; ++ch) {
        float v[16];
        if (nk > 0) {
          float v2[16];
          tmem_ld16(tbase + (uint32_t)(ch * 16), v);
          tmem_ld16(tbase + (uint32_t)(kAcc1 + ch * 16), v2);
#pragma unroll
          for (int k = 0; k < 16; ++k) v[k] = (v[k] + v2[k]) * ep.inv_nm;
        } else {
#pragma unroll
          for (int k = 0; k < 16; ++k) v[k] = 0.0f;
        }
        if (Tr) {
#pragma unroll
          for (int k = 0; k < 16; k += 4)
            if (ch * 16 + k < M)
              __stcs(reinterpret_cast<float4*>(Tr + ch * 16 + k),
                     make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]));
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
  }
  nrange = __reduce_add_sync(0xffffffffu, nrange);
  if (lane == 0 && nrange) atomicAdd(&status[ST_RANGE], nrange);
  if (lane == 0 && nover) atomicAdd(&status[ST_SEL], nover);
  if (lane == 0 && pair_count && npairs) atomicAdd(pair_count, npairs);
  if (tid == 0 && *abort_flag) atomicAdd(&status[ST_TIMEOUT], 1);
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 2)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kTmemCols));
}

// ------------------------------------------------------------------ backward
// Per tile of 32 atoms (the forward's tiles): the bins of the tile's
// occupied range in windows of 16; per window
//   B[(atom, c)][(bin, q)] = (1/N_m) sum_m dT[atom][c][m] c_bin[q][m]
// on the tensor cores (A = dE/dT rows from FP32, split in the stage by warps
// 4-7; B = the table window, bulk copies), then B goes through TMEM to shared
// memory and every pair of the window takes its 24 values for the chain rule
// to the forces and virial (one warp per atom, lanes over the sorted pairs the
// forward left: displacement and neighbor index).
constexpr int kWin = 16;                    // bins per window (N <= 128)
constexpr int kBsmAtom = kWin * 24 + 4;     // floats per atom in the window buffer

struct BwdCfg {
  int NP, nbp, stage;
  size_t smem;
};

__host__ __device__ inline BwdCfg bwd_cfg(const EnvParams& ep) {
  BwdCfg c;
  c.NP = round16(ep.M);
  c.nbp = (ep.ntypes * ep.n_int + 7) & ~7;
  c.stage = kPC * kABytes + kPC * kWin * 8 * 32;
  size_t st = (size_t)kNS * c.stage;
  const size_t bsm = (size_t)kAtoms * kBsmAtom * 4;
  if (st < bsm) st = bsm;
  c.smem = 128 + st + (size_t)kAtoms * c.nbp * 2;
  return c;
}

template <bool COMPACT>  // skip windows without a pair (several neighbor types)
__global__ void __launch_bounds__(kThreads, 2)
    k_tab_bwd_tc(int64_t ntile, TileMap tm, const float4* __restrict__ pairs,
                 const uint16_t* __restrict__ hist_in, const int2* __restrict__ range_in,
                 EnvParams ep,
                 const __nv_bfloat16* __restrict__ tabB, int scap, const float* __restrict__ dT,
                 unsigned long long* __restrict__ ffix, double* __restrict__ vir_part,
                 int32_t* __restrict__ status, double* __restrict__ vir_tile) {
  // a forward that gave up on a bounded wait left tiles without sorted pairs,
  // bin ends or ranges: nothing here may index through them (the call
  // reports DP_ERR_TIMEOUT)
  if (status[ST_TIMEOUT] != 0) return;
  const BwdCfg cf = bwd_cfg(ep);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  size_t st_bytes = (size_t)kNS * cf.stage;
  if (st_bytes < (size_t)kAtoms * kBsmAtom * 4) st_bytes = (size_t)kAtoms * kBsmAtom * 4;
  uint16_t* shist = (uint16_t*)(base + st_bytes);
  float* Bsm = (float*)base;  // aliases the stages between the MMAs of two windows
  __shared__ __align__(8) uint64_t s_full[kNS], s_empty[kNS], s_gen[kNS], s_acc;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  __shared__ int s_atom[kAtoms];
  __shared__ double s_vir[kThreads / 32][9];
  __shared__ double s_vt[kThreads / 32][9];  // this tile's virial per warp (vir_tile)
  __shared__ uint32_t s_wocc[kMaxOccWords];  // windows of the range with a pair
  volatile int* abort_flag = &s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nbins = ep.ntypes * ep.n_int, n_int = ep.n_int;
  const int M = ep.M, NP = cf.NP, nkc = NP / 16;
  const int NB8 = 8 * even_bins(nbins);
  const size_t blk = (size_t)NB8 * 16;
  const int64_t tabB_ti = tabB_elems(nbins, NP);

  if (tid == 0) {
    for (int s = 0; s < kNS; ++s) {
      mbar_init(&s_full[s], 1);
      mbar_init(&s_empty[s], 1);
      mbar_init(&s_gen[s], kRows);
    }
    mbar_init(&s_acc, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (lane < 9) s_vir[warp][lane] = 0.0;
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = s_tmem;

  int nbad = 0;
  uint32_t it = 0, acc_n = 0;
  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int ti = tile_type(tm, tile);
    {
      const int4* hi4 = reinterpret_cast<const int4*>(hist_in + (size_t)tile * kAtoms * cf.nbp);
      int4* hs = reinterpret_cast<int4*>(shist);
      for (int q = tid; q < kAtoms * cf.nbp / 8; q += kThreads) hs[q] = hi4[q];
      if (tid < kAtoms) s_atom[tid] = tile_atom(tm, ti, tile, tid);
    }
    const int2 rg = range_in[tile];
    const int kb0 = rg.x, nbt = 2 * rg.y;  // bins kb0 .. kb0 + nbt - 1 (even count)
    __syncthreads();
    // windows without a pair of any atom of the tile are skipped (by every
    // warp alike: nothing of them is pipelined)
    if (COMPACT) {
      const int nwin = (nbt + kWin - 1) / kWin;
      mark_occupied(shist, cf.nbp, nbins, kb0, kWin, nwin, s_wocc, warp, lane, kThreads / 32);
      __syncthreads();
    }
    float fxa[kAtoms / 8], fya[kAtoms / 8], fza[kAtoms / 8];
#pragma unroll
    for (int j = 0; j < kAtoms / 8; ++j) fxa[j] = fya[j] = fza[j] = 0.0f;
    float vl[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) vl[a] = 0.0f;
    for (int w0 = kb0; w0 < kb0 + nbt; w0 += kWin) {
      const int wi = (w0 - kb0) / kWin;
      if (COMPACT && !((s_wocc[wi >> 5] >> (wi & 31)) & 1u)) continue;
      const int wb = min(kWin, kb0 + nbt - w0);  // even
      const int Wr = wb * 8;                     // MMA N (a multiple of 16)
      // ---- B window = dT . table^T on the tensor cores
      if (warp == 0) {
        if (lane == 0) {
          const __nv_bfloat16* Bt = tabB + (size_t)ti * tabB_ti + (size_t)w0 * 8 * 16;
          uint32_t i = it;
          int kc = 0;
          for (; kc < nkc; ++kc, ++i) {
            const int s = i % kNS;
            const uint32_t u = i / kNS;
            if (u > 0 && !mbar_wait(&s_empty[s], (u - 1) & 1, abort_flag)) break;
            mbar_expect_tx(&s_full[s], kPC * Wr * 32);
            const uint32_t dst = smem_u32(base + (size_t)s * cf.stage + kPC * kABytes);
#pragma unroll
            for (int p = 0; p < kPC; ++p)
              bulk_g2s(dst + p * Wr * 32, Bt + ((size_t)kc * kPC + p) * blk, Wr * 32, &s_full[s]);
          }
          if (kc < nkc) {
            for (uint32_t j = (i - it) > (uint32_t)kNS ? i - kNS : it; j < i; ++j)
              mbar_wait(&s_full[j % kNS], (j / kNS) & 1, nullptr);
          }
        }
        __syncwarp();
      } else if (warp == 1) {
        if (lane == 0) {
          const uint32_t idesc = make_idesc_bf16(kRows, Wr);
          uint32_t i = it;
          for (int kc = 0; kc < nkc; ++kc, ++i) {
            const int s = i % kNS;
            const uint32_t u = i / kNS;
            if (!mbar_wait(&s_full[s], u & 1, abort_flag)) break;
            if (!mbar_wait(&s_gen[s], u & 1, abort_flag)) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            const uint32_t st0 = smem_u32(base + (size_t)s * cf.stage);
#pragma unroll
            for (int q = 0; q < kNPROD; ++q) {
              int pa, pb;
              prod_pieces(q, pa, pb);
              const uint64_t ad = make_desc(st0 + pa * kABytes, 128, 256);
              const uint64_t bd = make_desc(st0 + kPC * kABytes + pb * Wr * 32, 128, 256);
              const uint32_t dst = tmem + (q > 0 ? (uint32_t)kAcc1 : 0u);
              const uint32_t acc = (kc > 0 || q > 1) ? 1u : 0u;
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dst),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    smem_u32(&s_empty[s])));
          }
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                  smem_u32(&s_acc)));
        }
        __syncwarp();
      } else if (warp >= 4) {
        // A rows: thread r = (atom al, component c), 16 columns of dE/dT per chunk
        const int r = tid - 128, al = r >> 2, c = r & 3;
        const int atom = s_atom[al];
        const float* dr = atom >= 0 ? dT + (size_t)atom * 4 * M + (size_t)c * M : nullptr;
        // the next chunk's 16 values are loaded before this chunk's stage wait
        float4 nx[4];
        auto load16 = [&](int kc) {
#pragma unroll
          for (int k = 0; k < 16; k += 4) {
            const int col = kc * 16 + k;
            nx[k / 4] = (dr && col < M) ? __ldg(reinterpret_cast<const float4*>(dr + col))
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        };
        load16(0);
        uint32_t i = it;
        for (int kc = 0; kc < nkc; ++kc, ++i) {
          const int s = i % kNS;
          const uint32_t u = i / kNS;
          float x[16];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            x[4 * k] = nx[k].x;
            x[4 * k + 1] = nx[k].y;
            x[4 * k + 2] = nx[k].z;
            x[4 * k + 3] = nx[k].w;
          }
          if (kc + 1 < nkc) load16(kc + 1);
          if (u > 0 && !mbar_wait(&s_empty[s], (u - 1) & 1, abort_flag)) break;
          unsigned char* sa = base + (size_t)s * cf.stage;
#pragma unroll
          for (int kg = 0; kg < 2; ++kg) {
            __align__(16) __nv_bfloat16 pv[3][8];
            split8<kPC>(x + kg * 8, pv);
            const int o = (r >> 3) * 256 + kg * 128 + (r & 7) * 16;
#pragma unroll
            for (int p = 0; p < kPC; ++p)
              *reinterpret_cast<uint4*>(sa + p * kABytes + o) = *reinterpret_cast<const uint4*>(pv[p]);
          }
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
          mbar_arrive(&s_gen[s]);
        }
      }
      it += nkc;
      if (!mbar_wait(&s_acc, acc_n & 1, nullptr)) *abort_flag = 1;
      ++acc_n;
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      __syncthreads();
      if (*abort_flag) break;
      // ---- B window: TMEM -> shared memory [atom][bin][c * 6 + q] (times 1/N_m)
      {
        const int lg = warp & 3, half = warp >> 2;
        const int row_t = lg * 32 + lane;
        const int al = row_t >> 2, c = row_t & 3;
        const uint32_t tbase = tmem + ((uint32_t)(lg * 32) << 16);
        const int nch = Wr / 16;
        const int c_beg = half ? (nch + 1) / 2 : 0, c_end = half ? nch : (nch + 1) / 2;
        for (int ch = c_beg; ch < c_end; ++ch) {
          float v[16], v2[16];
          tmem_ld16(tbase + (uint32_t)(ch * 16), v);
          tmem_ld16(tbase + (uint32_t)(kAcc1 + ch * 16), v2);
#pragma unroll
          for (int hb = 0; hb < 2; ++hb) {
            float* dst = Bsm + al * kBsmAtom + (2 * ch + hb) * 24 + c * 6;
#pragma unroll
            for (int q = 0; q < 6; ++q) dst[q] = (v[hb * 8 + q] + v2[hb * 8 + q]) * ep.inv_nm;
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n");
      __syncthreads();
      // ---- pairs of the window: chain rule to the forces and virial
      const int wend = min(w0 + wb, nbins);  // bins w0 .. wend - 1 exist
      // the window's pairs of the warp's four atoms as one range t = 0 ..
      // total - 1 (atom j from the prefix counts cs, sorted index k), so the
      // lanes stay busy across the atoms; the next pair is loaded while the
      // current one is computed
      const int al0 = warp * (kAtoms / 8);
      int kb0 = 0, kb1 = 0, kb2 = 0, kb3 = 0, cs1, cs2, cs3, total;
      {
        int n4[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint16_t* hist = shist + (al0 + j) * cf.nbp;
          const bool live = s_atom[al0 + j] >= 0;
          const int b = live ? bin_begin16(hist, w0) : 0;
          n4[j] = live ? hist[wend - 1] - b : 0;
          if (j == 0) kb0 = b;
          if (j == 1) kb1 = b;
          if (j == 2) kb2 = b;
          if (j == 3) kb3 = b;
        }
        cs1 = n4[0];
        cs2 = cs1 + n4[1];
        cs3 = cs2 + n4[2];
        total = cs3 + n4[3];
      }
      auto locate = [&](int t, int& j, int& k) {
        j = (t >= cs1) + (t >= cs2) + (t >= cs3);
        const int kbj = j == 0 ? kb0 : j == 1 ? kb1 : j == 2 ? kb2 : kb3;
        const int csj = j == 0 ? 0 : j == 1 ? cs1 : j == 2 ? cs2 : cs3;
        k = kbj + (t - csj);
      };
      const float4* pr_tile = pairs + (size_t)tile * kAtoms * scap;
      float4 nxt = make_float4(0.f, 0.f, 0.f, 0.f);
      if (lane < total) {
        int j, k;
        locate(lane, j, k);
        nxt = pr_tile[(size_t)(al0 + j) * scap + k];
      }
      for (int t = lane; t < total; t += 32) {
        const float4 q4 = nxt;
        int jq, kq;
        locate(t, jq, kq);
        if (t + 32 < total) {
          int jn2, kn2;
          locate(t + 32, jn2, kn2);
          nxt = pr_tile[(size_t)(al0 + jn2) * scap + kn2];
        }
        const int al = al0 + jq;
        const uint16_t* hist = shist + al * cf.nbp;
        // the pair's bin: the first in [w0, wend) whose end exceeds kq
        int b = w0, bh = wend - 1;
        while (b < bh) {
          const int mid = (b + bh) >> 1;
          if (hist[mid] > kq) bh = mid;
          else b = mid + 1;
        }
        const float dx = q4.x, dy = q4.y, dz = q4.z;
        const int jn = __float_as_int(q4.w);
        const int tj = b / n_int, th = b - tj * n_int;
        const float r2 = dx * dx + dy * dy + dz * dz;
        Pair P;
        pair_geom(ep, dx, dy, dz, r2, tj, P);
        const float u = interval_u(ep, P.s, th);  // the sort's interval
        const float* Bk = Bsm + al * kBsmAtom + (b - w0) * 24;
        float Bv[24];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const float4 t4 = reinterpret_cast<const float4*>(Bk)[q];
          Bv[4 * q] = t4.x;
          Bv[4 * q + 1] = t4.y;
          Bv[4 * q + 2] = t4.z;
          Bv[4 * q + 3] = t4.w;
        }
        float gR[4], dgu[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float* bb = Bv + c * 6;
          gR[c] = fmaf(fmaf(fmaf(fmaf(fmaf(bb[5], u, bb[4]), u, bb[3]), u, bb[2]), u, bb[1]), u, bb[0]);
          dgu[c] = fmaf(fmaf(fmaf(fmaf(5.0f * bb[5], u, 4.0f * bb[4]), u, 3.0f * bb[3]), u,
                             2.0f * bb[2]),
                        u, bb[1]);
        }
        const float ux = P.dx * P.ir, uy = P.dy * P.ir, uz = P.dz * P.ir;
        const float s = P.s;
        const float gs =
            interval_du_ds(ep, th) * s * (dgu[0] + ux * dgu[1] + uy * dgu[2] + uz * dgu[3]);
        const float a0 = gR[0] + gs;
        const float dot = gR[1] * ux + gR[2] * uy + gR[3] * uz;
        const float sor = s * P.ir;
        const float coef = P.dsdr * (a0 + dot) - sor * dot;
        float gx = coef * ux + sor * gR[1];
        float gy = coef * uy + sor * gR[2];
        float gz = coef * uz + sor * gR[3];
        if (!(isfinite(gx) && isfinite(gy) && isfinite(gz)) || fabsf(gx) > 4.0e6f ||
            fabsf(gy) > 4.0e6f || fabsf(gz) > 4.0e6f) {
          ++nbad;
          gx = gy = gz = 0.0f;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (jq == j) {
            fxa[j] += gx;
            fya[j] += gy;
            fza[j] += gz;
          }
        vl[0] -= dx * gx;
        vl[1] -= dx * gy;
        vl[2] -= dx * gz;
        vl[3] -= dy * gx;
        vl[4] -= dy * gy;
        vl[5] -= dy * gz;
        vl[6] -= dz * gx;
        vl[7] -= dz * gy;
        vl[8] -= dz * gz;
        unsigned long long* fj = ffix + (size_t)jn * 3;
        atomicAdd(fj + 0, (unsigned long long)(-__float2ll_rn(gx * DP_FSCALE_F)));
        atomicAdd(fj + 1, (unsigned long long)(-__float2ll_rn(gy * DP_FSCALE_F)));
        atomicAdd(fj + 2, (unsigned long long)(-__float2ll_rn(gz * DP_FSCALE_F)));
      }
      // the window buffer is read before the next window's bulk copies land there
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      __syncthreads();
    }
    if (*abort_flag) break;
    // the centres' own forces: lane partials summed across the warp in FP64
#pragma unroll
    for (int j = 0; j < kAtoms / 8; ++j) {
      const int atom = s_atom[warp * (kAtoms / 8) + j];
      double red[3] = {fxa[j], fya[j], fza[j]};
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
        for (int a = 0; a < 3; ++a) red[a] += __shfl_xor_sync(0xffffffffu, red[a], o);
      if (lane == 0 && atom >= 0) {
        unsigned long long* fi = ffix + (size_t)atom * 3;
        atomicAdd(fi + 0, (unsigned long long)__double2ll_rn(red[0] * DP_FSCALE));
        atomicAdd(fi + 1, (unsigned long long)__double2ll_rn(red[1] * DP_FSCALE));
        atomicAdd(fi + 2, (unsigned long long)__double2ll_rn(red[2] * DP_FSCALE));
      }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
      for (int a = 0; a < 9; ++a) vl[a] += __shfl_xor_sync(0xffffffffu, vl[a], o);
    if (lane < 9) {
      float vv = vl[0];
#pragma unroll
      for (int a = 1; a < 9; ++a) vv = lane == a ? vl[a] : vv;
      if (vir_tile) s_vt[warp][lane] = (double)vv;
      else s_vir[warp][lane] += (double)vv;
    }
    __syncthreads();  // shist and s_atom are refilled by the next tile
    if (vir_tile && tid < 9) {
      // one row per tile (several systems in one launch: tiles never span two)
      double v = 0.0;
#pragma unroll
      for (int w = 0; w < kThreads / 32; ++w) v += s_vt[w][tid];
      vir_tile[(size_t)tile * 9 + tid] = v;
    }
  }
  if (lane < 9) vir_part[((size_t)blockIdx.x * (kThreads / 32) + warp) * 9 + lane] = s_vir[warp][lane];
  nbad = __reduce_add_sync(0xffffffffu, nbad);
  if (lane == 0 && nbad) atomicAdd(&status[ST_NONFINITE], nbad);
  if (tid == 0 && *abort_flag) atomicAdd(&status[ST_TIMEOUT], 1);
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 2)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kTmemCols));
}

// ------------------------------------------------------------------ table gradient
// dE/dc[ti][b][q][m] = (1/N_m) sum over the rows (atom i of type ti, c) of
//   C[(i,c)][(b,q)] dE/dT_i[c][m],   C[(i,c)][(b,q)] = sum_{j in bin b} R_jc u_j^q
// (T is linear in the table: the forward's contraction read the other way).
// Per tile of the forward (its sorted displacements, bin ends and bin
// range): the tile's dE/dT rows in shared memory; per window of 16 bins the
// window's C is recomputed from the sorted displacements (the arithmetic of
// the forward's sort) and multiplied with dE/dT on the CUDA cores; the
// products go into the CTA's own FP32 partial (read-modify-write, no
// atomics).  A second kernel sums the partials over the CTAs in FP64, in CTA
// order, so the result is deterministic.
constexpr int kGWin = 16;            // bins per window
constexpr int kGCs = kGWin * 6 + 4;  // floats per row of the C window

__host__ __device__ inline int grad_mp(int M) { return (M + 3) / 4 * 4; }
__host__ __device__ inline size_t grad_smem(const EnvParams& ep) {
  const int nbp = (ep.ntypes * ep.n_int + 7) & ~7;
  return 128 + (size_t)kRows * grad_mp(ep.M) * 4 + (size_t)kRows * kGCs * 4 +
         (size_t)kAtoms * nbp * 2;
}

__global__ void __launch_bounds__(kThreads, 1)
    k_tab_grad_tc(int64_t ntile, TileMap tm, const float4* __restrict__ pairs,
                  const uint16_t* __restrict__ hist_in, const int2* __restrict__ range_in,
                  EnvParams ep, int scap, const float* __restrict__ dT, float* __restrict__ part) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  const int M = ep.M, MP = grad_mp(M);
  const int nbins = ep.ntypes * ep.n_int;
  const int nbp = (nbins + 7) & ~7;
  float* dTs = (float*)base;                   // [kRows][MP]
  float* Cs = dTs + (size_t)kRows * MP;        // [kRows][kGCs]
  uint16_t* shist = (uint16_t*)(Cs + (size_t)kRows * kGCs);  // [kAtoms][nbp]
  __shared__ int s_atom[kAtoms];
  const int tid = threadIdx.x;
  float* part_cta = part + (size_t)blockIdx.x * ep.ntypes * nbins * 6 * M;

  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int ti = tile_type(tm, tile);
    {
      const int4* hi4 = reinterpret_cast<const int4*>(hist_in + (size_t)tile * kAtoms * nbp);
      int4* hs = reinterpret_cast<int4*>(shist);
      for (int q = tid; q < kAtoms * nbp / 8; q += kThreads) hs[q] = hi4[q];
      if (tid < kAtoms) s_atom[tid] = tile_atom(tm, ti, tile, tid);
    }
    __syncthreads();
    for (int q = tid; q < kRows * M; q += kThreads) {
      const int r = q / M, m = q - r * M;
      const int atom = s_atom[r >> 2];
      dTs[r * MP + m] = atom >= 0 ? dT[(size_t)atom * 4 * M + (size_t)(r & 3) * M + m] : 0.0f;
    }
    const int2 rg = range_in[tile];
    const int kb0 = rg.x, nbt = 2 * rg.y;
    for (int w0 = kb0; w0 < kb0 + nbt; w0 += kGWin) {
      const int wb = min(kGWin, kb0 + nbt - w0);
      {
        // C window: thread (row r = (al, c), half hh) builds 8 bins of its row
        const int r = tid & (kRows - 1), hh = tid >> 7;
        const int al = r >> 2, c = r & 3;
        const int atom = s_atom[al];
        const uint16_t* hist = shist + al * nbp;
        const float4* pr = pairs + ((size_t)tile * kAtoms + al) * scap;
        for (int j = hh * 8; j < hh * 8 + 8; ++j) {
          const int b = w0 + j;
          float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
          if (j < wb && b < nbins && atom >= 0) {
            const int tj = b / ep.n_int;
            const int kend = hist[b];
            for (int k = bin_begin16(hist, b); k < kend; ++k) {
              const float4 q4 = pr[k];
              const float r2 = q4.x * q4.x + q4.y * q4.y + q4.z * q4.z;
              Pair P;
              pair_geom(ep, q4.x, q4.y, q4.z, r2, tj, P);
              const float d = c == 1 ? P.dx : (c == 2 ? P.dy : P.dz);
              const float Rc = c == 0 ? P.s : P.s * d * P.ir;
              float up = Rc;
#pragma unroll
              for (int t = 0; t < 6; ++t) {
                acc[t] += up;
                up *= P.u;
              }
            }
          }
#pragma unroll
          for (int t = 0; t < 6; ++t) Cs[r * kGCs + j * 6 + t] = acc[t];
        }
      }
      __syncthreads();
      {
        // the window's products: thread (column m, half hh) owns 48 (b, q)
        const int m = tid & (kRows - 1), hh = tid >> 7;
        if (m < M) {
          float acc[48];
#pragma unroll
          for (int j = 0; j < 48; ++j) acc[j] = 0.0f;
          for (int r = 0; r < kRows; ++r) {
            const float a = dTs[r * MP + m];
            const float4* cr = reinterpret_cast<const float4*>(Cs + r * kGCs + hh * 48);
#pragma unroll
            for (int v = 0; v < 12; ++v) {
              const float4 c4 = cr[v];
              acc[4 * v] = fmaf(c4.x, a, acc[4 * v]);
              acc[4 * v + 1] = fmaf(c4.y, a, acc[4 * v + 1]);
              acc[4 * v + 2] = fmaf(c4.z, a, acc[4 * v + 2]);
              acc[4 * v + 3] = fmaf(c4.w, a, acc[4 * v + 3]);
            }
          }
#pragma unroll
          for (int j = 0; j < 48; ++j) {
            const int bq = hh * 48 + j, b = w0 + bq / 6;
            if (bq < wb * 6 && b < nbins)
              part_cta[((size_t)(ti * nbins + b) * 6 + bq % 6) * M + m] += acc[j];
          }
        }
      }
      __syncthreads();
    }
  }
}

// out[e] = (1/N_m) sum over the CTAs (in order) of part[cta][e]
__global__ void k_tab_grad_reduce(int nct, int64_t n, const float* __restrict__ part,
                                  float inv_nm, double* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  double s = 0.0;
  for (int k = 0; k < nct; ++k) s += (double)part[(size_t)k * n + e];
  out[e] = s * (double)inv_nm;
}

std::atomic<int> g_sms{0};
int sm_count() {
  if (!g_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    g_sms = v > 0 ? v : 1;
  }
  return g_sms;
}

int stage_cap_tc(const EnvParams& ep) { return scap_of(ep); }

int tc_grid() { return 2 * sm_count(); }

}  // namespace

int64_t tab_tc_elems(const EnvParams& ep) {
  const int nbins = ep.ntypes * ep.n_int, NP = round16(ep.M);
  const int64_t f = tabF_elems(nbins, NP), b = tabB_elems(nbins, NP);
  return (f > b ? f : b) * ep.ntypes;
}

int tab_tc_build(cudaStream_t st, const float* table, const EnvParams& ep, __nv_bfloat16* tabF,
                 __nv_bfloat16* tabB) {
  if (ep.M > 128 || ep.M % 4) return -1;
  const int nbins = ep.ntypes * ep.n_int, NP = round16(ep.M);
  const int64_t nf = (int64_t)ep.ntypes * tabF_elems(nbins, NP) / kPC;
  const int64_t nb = (int64_t)ep.ntypes * tabB_elems(nbins, NP) / kPC;
  DP_LAUNCHED(2);
  k_tile_tabF<<<(int)((nf + 255) / 256), 256, 0, st>>>(table, ep.ntypes, nbins, ep.M, NP, tabF);
  k_tile_tabB<<<(int)((nb + 255) / 256), 256, 0, st>>>(table, ep.ntypes, nbins, ep.M, NP, tabB);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int64_t tab_tc_scratch_floats(const EnvParams& ep) {
  return (int64_t)tc_grid() * 5 * kAtoms * stage_cap_tc(ep);
}

int launch_tab_fwd_tc(cudaStream_t st, const TileMap& tm, const float4* off, const uint32_t* nlist,
                      const int32_t* nn, int cap, const CellGeom& g, const EnvParams& ep,
                      const __nv_bfloat16* tabF, float* scratch, float4* pairs_out,
                      uint16_t* hist_out, int2* range_out, float* T, int32_t* status,
                      unsigned long long* pair_count, const int32_t* sys_of,
                      const int32_t* sys_base, const float4* sys_edge, long long gen_wait_limit) {
  if (ep.M > 128 || ep.M % 4 || ep.M < 16) return -1;
  if (gen_wait_limit < 0) gen_wait_limit = kSpinLimit;
  if (tm.ntypes < 1 || tm.ntypes > DP_MAXT || tm.ntypes != ep.ntypes) return -1;
  if (((uintptr_t)tabF & 15) || ((uintptr_t)T & 15)) return -1;
  if (tab_tc_supported(ep)) return -1;
  const int64_t ntile = tm.tile_off[tm.ntypes];
  if (ntile <= 0) return 0;
  const FwdCfg cf = fwd_cfg(ep);
  if (cf.smem > 113 * 1024) return -1;  // two CTAs per SM
  const bool compact = ep.ntypes > 1;
  auto kern = compact ? k_tab_fwd_tc<true> : k_tab_fwd_tc<false>;
  static std::atomic<size_t> set[2] = {{0}, {0}};  // launches from several host threads
  if (cf.smem > 48 * 1024 && cf.smem > set[compact]) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)cf.smem) != cudaSuccess)
      return -3;
    set[compact] = cf.smem;
  }
  const int grid = (int)(ntile < tc_grid() ? ntile : tc_grid());
  DP_LAUNCHED(1);
  kern<<<grid, kThreads, cf.smem, st>>>(ntile, tm, off, nlist, nn, cap, g, ep, tabF,
                                        stage_cap_tc(ep), scratch, pairs_out, hist_out,
                                        range_out, T, status, pair_count, sys_of, sys_base,
                                        sys_edge, gen_wait_limit);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int64_t tab_tc_slots() { return (int64_t)tc_grid() * (kThreads / 32); }

int launch_tab_bwd_tc(cudaStream_t st, const TileMap& tm, const float4* pairs,
                      const uint16_t* hist,
                      const int2* range, const EnvParams& ep, const __nv_bfloat16* tabB,
                      const float* dT, unsigned long long* ffix, double* vir_part, int vir_slots,
                      int32_t* status, double* vir_tile) {
  if (ep.M > 128 || ep.M % 4 || ep.M < 16) return -1;
  if (tm.ntypes < 1 || tm.ntypes > DP_MAXT || tm.ntypes != ep.ntypes) return -1;
  if (((uintptr_t)tabB & 15) || ((uintptr_t)dT & 15) || ((uintptr_t)hist & 15)) return -1;
  if (vir_slots < tab_tc_slots()) return -1;
  const int64_t ntile = tm.tile_off[tm.ntypes];
  if (ntile <= 0) return 0;
  const BwdCfg cf = bwd_cfg(ep);
  if (cf.smem > 113 * 1024) return -1;  // two CTAs per SM
  const bool compact = ep.ntypes > 1;
  auto kern = compact ? k_tab_bwd_tc<true> : k_tab_bwd_tc<false>;
  static std::atomic<size_t> set[2] = {{0}, {0}};  // launches from several host threads
  if (cf.smem > 48 * 1024 && cf.smem > set[compact]) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)cf.smem) != cudaSuccess)
      return -3;
    set[compact] = cf.smem;
  }
  // every slot is written (grid = the full persistent grid, idle CTAs write zeros)
  DP_LAUNCHED(1);
  kern<<<tc_grid(), kThreads, cf.smem, st>>>(ntile, tm, pairs, hist, range, ep, tabB,
                                             stage_cap_tc(ep), dT, ffix, vir_part, status,
                                             vir_tile);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ------------------------------------------------------------------ table gradient
int64_t tab_grad_part_floats(const EnvParams& ep) {
  return (int64_t)sm_count() * ep.ntypes * ep.ntypes * ep.n_int * 6 * ep.M;
}

int launch_tab_grad_tc(cudaStream_t st, const TileMap& tm, const float4* pairs,
                       const uint16_t* hist, const int2* range, const EnvParams& ep,
                       const float* dT, float* part, double* grad) {
  if (ep.M > 128 || ep.M % 4 || ep.M < 16) return -1;
  if (tm.ntypes < 1 || tm.ntypes > DP_MAXT || tm.ntypes != ep.ntypes) return -1;
  if (((uintptr_t)hist & 15) || ((uintptr_t)part & 15)) return -1;
  const int64_t n = (int64_t)ep.ntypes * ep.ntypes * ep.n_int * 6 * ep.M;
  const int64_t ntile = tm.tile_off[tm.ntypes];
  const size_t smem = grad_smem(ep);
  if (smem > 225 * 1024) return -1;
  static std::atomic<size_t> set{0};  // launches from several host threads
  if (smem > 48 * 1024 && smem > set) {
    if (cudaFuncSetAttribute(k_tab_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return -3;
    set = smem;
  }
  const int grid = sm_count();
  if (cudaMemsetAsync(part, 0, sizeof(float) * (size_t)grid * n, st) != cudaSuccess) return -3;
  DP_LAUNCHED(2);
  if (ntile > 0)
    k_tab_grad_tc<<<grid, kThreads, smem, st>>>(ntile, tm, pairs, hist, range, ep,
                                                stage_cap_tc(ep), dT, part);
  k_tab_grad_reduce<<<(int)((n + 255) / 256), 256, 0, st>>>(grid, n, part, ep.inv_nm, grad);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int64_t tab_tc_pair_elems(const EnvParams& ep, int64_t ntile) {
  return ntile * kAtoms * stage_cap_tc(ep);
}
int64_t tab_tc_hist_elems(const EnvParams& ep, int64_t ntile) {
  return ntile * kAtoms * ((ep.ntypes * ep.n_int + 7) & ~7);
}

int tab_tc_supported(const EnvParams& ep) {
  if (ep.M > 128 || ep.M % 4 || ep.M < 16) return -1;
  // the occupancy masks: at most 32 * kMaxOccWords chunks of two bins
  if (ep.ntypes * ep.n_int + 2 > 2 * 32 * kMaxOccWords) return -2;
  if (fwd_cfg(ep).smem > 113 * 1024 || bwd_cfg(ep).smem > 113 * 1024) return -2;

  return 0;
}
