// Internal declarations shared by the CUDA kernels and the C-ABI runtime.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dp.h"

#define DP_MAXT 8
#define DP_MAXFIT 6

// Number of kernels this library has launched in the process (all threads).
extern unsigned long long g_dp_launches;
extern thread_local unsigned long long g_dp_launches_tl;  // this thread's share
#define DP_LAUNCHED(k)                                                               \
  (__atomic_fetch_add(&g_dp_launches, (unsigned long long)(k), __ATOMIC_RELAXED),    \
   g_dp_launches_tl += (unsigned long long)(k))

// Per-call device status words (int32).  Kernels only ever add / max into them.
enum {
  ST_SEL = 0,        // atoms with more neighbors of one type within rc than sel[t]
  ST_RANGE = 1,      // pairs with s outside [0, n*h]
  ST_NONFINITE = 2,  // non-finite per-atom energies / forces
  ST_SKIN = 3,       // atoms displaced more than skin/2 since the last rebuild
  ST_MAXLIST = 4,    // largest list length seen (may exceed the capacity)
  ST_LISTOVF = 5,    // atoms whose list did not fit the capacity
  ST_BADTYPE = 6,    // atoms with a type index outside the type map
  ST_TIMEOUT = 7,    // bounded device waits that gave up
  ST_NWORDS = 16
};

// Fixed-point force accumulators: F = int64 * 2^-40 eV/A.  Integer adds are
// associative, so the atomics give the same bits in any order.
#define DP_FSCALE 1099511627776.0 /* 2^40 */
#define DP_FSCALE_F 1099511627776.0f
#define DP_FINV (1.0 / 1099511627776.0)

// Geometry of the cell grid used for a neighbor list.  Cells have edge >=
// rlist; each atom carries its FP32 offset from the centre of the cell it
// was binned into at the last rebuild, so a pair displacement is
//   r_ij = (off_j - off_i) + o * edge,  o in {-1,0,1}^3 the stencil offset.
struct CellGeom {
  double L[3];
  double edge[3];
  float edgef[3];
  int nc[3];
  long long ncell;
};

// Smooth-switch / table parameters in FP32 for the pair kernels.
struct EnvParams {
  float rc2, rc, rcs, inv_w;  // inv_w = 1/(rc - rcs)
  float inv_h, h, smax;       // table step and domain end (the last node)
  float s_fine, inv_H;        // end of the step-h region; 1/width beyond it
  float inv_nm;               // 1/N_m (N_m = sum of sel)
  int n_int;                  // table intervals
  int n_fine;                 // of them of width h (the rest, of width H)
  int M;                      // embedding width
  int ntypes;                 // model types
};

// ---------------------------------------------------------------- neighbors
void launch_wrap_bin(cudaStream_t st, int64_t n, double* x, const CellGeom& g, int32_t* cellc,
                     int32_t* cell_count);
void launch_scan(cudaStream_t st, const int32_t* count, int32_t* start, long long ncell);
void launch_scatter(cudaStream_t st, int64_t n, const int32_t* cellc, const int32_t* start,
                    int32_t* fill, int32_t* cell_atoms_unsorted);
void launch_cell_sort(cudaStream_t st, long long ncell, const int32_t* start,
                      const int32_t* unsorted, int32_t* sorted);
void launch_mirror(cudaStream_t st, int64_t n, const double* x, const int32_t* cellc,
                   const int32_t* types, const CellGeom& g, float4* off);
// several systems: atom i uses the cell grid geoms[sys_of[i]] (device array)
void launch_mirror_batch(cudaStream_t st, int64_t n, const double* x, const int32_t* cellc,
                         const int32_t* types, const int32_t* sys_of, const CellGeom* geoms,
                         float4* off);
void launch_build_list(cudaStream_t st, int64_t n, const double* x, const int32_t* cellc,
                       const float4* off, const int32_t* cell_start, const int32_t* cell_atoms,
                       const CellGeom& g, double rlist, float rc2, int ntypes, const int32_t* sel,
                       int cap, uint32_t* nlist, int32_t* nn, int32_t* status);

// ---------------------------------------------------------------- embedding
// FP64 forward-mode evaluation of every embedding net at the nodes (k*h for
// k <= n_fine, then steps of H) and the quintic fit per interval; writes FP32
// [npair][n_int][6][M] with the coefficients of the normalised local
// variable u = (s - x_k)/w_k.
int table_build(cudaStream_t st, const double* emb64, const int64_t* emb_off, int n_emb,
                const int* emb_w, int npair, double h, int n_int, int n_fine, double H,
                float* table_out);
int launch_tab_fwd(cudaStream_t st, int64_t n, const float4* off, const uint32_t* nlist,
                   const int32_t* nn, int cap, const CellGeom& g, const EnvParams& ep,
                   const float* table, float* T, int32_t* status,
                   unsigned long long* pair_count);
int launch_tab_bwd(cudaStream_t st, int64_t n, const float4* off, const uint32_t* nlist,
                   const int32_t* nn, int cap, const CellGeom& g, const EnvParams& ep,
                   const float* table, const float* dT, unsigned long long* ffix,
                   double* vir_part, int vir_slots, int32_t* status);
int tab_kernel_slots(int64_t n);  // number of virial partial slots the bwd kernel writes

// Tensor-core tabulated embedding (tcgen05, FP32-accurate 3-piece BF16
// operands): atoms grouped by model type in tiles of 32; tile t of type ti
// holds atoms idx[atom_off[ti] + 32 (t - tile_off[ti]) + 0..31] (idx == NULL:
// the positions themselves), the last tile of a type padded.
struct TileMap {
  int ntypes;
  int64_t tile_off[DP_MAXT + 1];
  int64_t atom_off[DP_MAXT];
  int64_t atom_cnt[DP_MAXT];
  const int32_t* idx;
};
// BF16 pieces of the table in the two pre-tiled operand layouts (forward:
// N = M columns x K = (interval, power); backward: N = (interval, power) x
// K = M); elements per centre type of each
int64_t tab_tc_elems(const EnvParams& ep);
int tab_tc_build(cudaStream_t st, const float* table, const EnvParams& ep, __nv_bfloat16* tabF,
                 __nv_bfloat16* tabB);
int64_t tab_tc_scratch_floats(const EnvParams& ep);  // scratch one launch needs
// the forward leaves, per tile, the sorted pairs (dx, dy, dz, neighbor index)
// [tile][32][N_m + 32 rounded], the bin ends (uint16) [tile][32][bins rounded
// to 8] and
// (first bin, chunks of two bins); the backward reads them
int64_t tab_tc_pair_elems(const EnvParams& ep, int64_t ntile);
int64_t tab_tc_hist_elems(const EnvParams& ep, int64_t ntile);
int64_t tab_tc_slots();  // virial partial slots the backward writes
// 0 if the tensor-core embedding can run this shape; -1 embedding width (M <=
// 128, M % 4 == 0), -2 too many table bins for the shared-memory histograms
int tab_tc_supported(const EnvParams& ep);
// dE/d(table coefficients) [ntypes][ntypes][n_int][6][M] (FP64, the layout of
// the device table) from the forward's sorted pairs, bin ends and ranges and
// dE/dT; part: tab_grad_part_floats floats of per-CTA partials
int64_t tab_grad_part_floats(const EnvParams& ep);
int launch_tab_grad_tc(cudaStream_t st, const TileMap& tm, const float4* pairs,
                       const uint16_t* hist, const int2* range, const EnvParams& ep,
                       const float* dT, float* part, double* grad);
// Several systems in one launch: sys_of [atoms] -> system, sys_base [systems]
// first atom, sys_edge [systems] cell edges (x, y, z, 0); the neighbor lists
// then hold system-local indices.  All NULL: one system.
int launch_tab_fwd_tc(cudaStream_t st, const TileMap& tm, const float4* off, const uint32_t* nlist,
                      const int32_t* nn, int cap, const CellGeom& g, const EnvParams& ep,
                      const __nv_bfloat16* tabF, float* scratch, float4* pairs_out,
                      uint16_t* hist_out, int2* range_out, float* T, int32_t* status,
                      unsigned long long* pair_count, const int32_t* sys_of = nullptr,
                      const int32_t* sys_base = nullptr, const float4* sys_edge = nullptr,
                      long long gen_wait_limit = -1);
// vir_tile != NULL: the virial as one FP64 row of 9 per tile (several systems
// in one launch, tiles padded per system) instead of the per-slot partials
int launch_tab_bwd_tc(cudaStream_t st, const TileMap& tm, const float4* pairs, const uint16_t* hist,
                      const int2* range, const EnvParams& ep, const __nv_bfloat16* tabB,
                      const float* dT, unsigned long long* ffix, double* vir_part, int vir_slots,
                      int32_t* status, double* vir_tile = nullptr);

// plain untabulated embedding (the comparator of the tabulation), FP32
int plain_kernel_slots(int64_t n);
size_t plain_net_bytes();
bool plain_net_fill(void* rec, const float* W0, const float* b0, const float* W1, const float* b1,
                    const float* W2, const float* b2, const float* W1T, const float* W2T);
int launch_plain_fwd(cudaStream_t st, int64_t n, const float4* off, const uint32_t* nlist,
                     const int32_t* nn, int cap, const CellGeom& g, const EnvParams& ep,
                     const void* nets, int d1, float* T, unsigned long long* pair_count);
int launch_plain_bwd(cudaStream_t st, int64_t n, const float4* off, const uint32_t* nlist,
                     const int32_t* nn, int cap, const CellGeom& g, const EnvParams& ep,
                     const void* nets, int d1, const float* dT, unsigned long long* ffix,
                     double* vir_part, int vir_slots, int32_t* status);
// dE/d(embedding-net parameters) of type pair (ti, tj) added into grad (FP64,
// per layer a [(win + 1)][wout] block: W rows then b; win_0 = 1) from dE/dT;
// part: plain_wgrad_ctas() x plain_wgrad_params() floats
int plain_wgrad_params(int d1, int M);
int plain_wgrad_ctas();
int launch_plain_wgrad(cudaStream_t st, int64_t n, const float4* off, const uint32_t* nlist,
                       const int32_t* nn, int cap, const CellGeom& g, const EnvParams& ep,
                       const void* nets, int d1, const float* dT, int ti, int tj, float* part,
                       double* grad);

// ---------------------------------------------------------------- fitting
struct FitNet {           // one centre type, FP32 device pointers
  int nl;                 // hidden layers
  int win[DP_MAXFIT];     // input width of layer k
  int wout[DP_MAXFIT];    // output width of layer k
  int shortcut[DP_MAXFIT];
  const float* W[DP_MAXFIT];   // [win][wout]
  const float* WT[DP_MAXFIT];  // [wout][win]
  const float* b[DP_MAXFIT];
  const float* w_out;          // [wout[nl-1]]
  float b_out;
  const float4* tanh_tab;      // Sec. 3.5 tanh table [1024] (a0, a1, a2, 0), or NULL
};
struct FitScratch {
  int64_t rows;  // capacity in atoms
  float* D;      // [rows][din]
  float* dD;     // [rows][din]
  float* t[DP_MAXFIT];  // activation derivatives (for the backward)
  float* z[DP_MAXFIT];
  float* gz;     // [rows][wmax]
  float* gp;     // [rows][wmax]
  float* gz2;    // [rows][wmax]
};
// E_i and dE/dT for atoms [0, n) of one centre type listed in idx (or all
// atoms when idx == NULL), FP32 CUDA-core path.
// With fg != NULL the same pass also adds dE/d(parameters) of this type's net
// into fg->g (FP64; per layer k a [(win_k + 1)][wout_k] block, W_k rows then
// b_k, then [(w_last + 1)]: w_out, b_out), through FP32 partials in fg->part.
struct FitGrad {
  double* g;
  float* part;
  int64_t part_floats;
};
int fit_simt(cudaStream_t st, int64_t n, const int32_t* idx, const FitNet& net, int M, int m_lt,
             const float* T, float* dT, double* e_atom, const FitScratch& s,
             const FitGrad* fg = nullptr);
// floats of fg->part that fit_simt needs for a net and chunk size
int64_t fit_grad_part_floats(const FitNet& net, int din, int64_t rows);

// Tensor-core (tcgen05, 16-bit operands, FP32 accumulate) fitting stage.  Each
// operand has 1 BF16 piece (BF16 mode), an FP16 pair x s = h + l (FP32-
// accurate, three piece products; s a power of two from a bound of |x|) or
// 3 BF16 pieces x = h + m + l (FP32-accurate, six piece products).  Operands
// are kept pre-tiled: per (row tile, 16-wide K chunk) one contiguous block
// holding all pieces in the tensor core's no-swizzle K-major layout (weights
// in tiles of N <= 256 rows, activations in tiles of 128 rows).
struct FitNetTC {
  int nl;
  int win[DP_MAXFIT], wout[DP_MAXFIT], shortcut[DP_MAXFIT];
  const __nv_bfloat16* WTh[DP_MAXFIT];  // tiled pieces of W^T [wout][win]: forward B operand
  const __nv_bfloat16* Wh[DP_MAXFIT];   // tiled pieces of W [win][wout]: backward B operand
  // FP16-pair scales (powers of two; 1 in the BF16 modes): of the pieces of
  // W^T and W of layer k, of the layer outputs z_k (the next layer's A) and
  // of the gradients dE/d(pre-activation) of layer k (the backward's A)
  float s_wt[DP_MAXFIT], s_w[DP_MAXFIT], s_z[DP_MAXFIT], s_g[DP_MAXFIT];
  const float* b[DP_MAXFIT];
  const float* w_out;
  float b_out;
  const float4* tanh_tab;  // Sec. 3.5 tanh table, or NULL
};
struct FitScratchTC {
  int64_t rows;                  // rows per chunk (a multiple of 128)
  int wmax;
  // FP32 arrays in the row-tile-chunked layout (per 128-row tile and
  // 16-column chunk a block of 128 x 16 floats)
  float* t[DP_MAXFIT];  // [rows][wout[k]] tanh values (table mode: derivatives)
  float* z[DP_MAXFIT];  // [rows][wout[k]] layer outputs (the next hidden layer's A operand)
  float* gz;              // [rows][wmax] dE/dz
  __nv_bfloat16* zh;      // tiled pieces of the last hidden z (the last layer's A operand)
  __nv_bfloat16* gph[2];  // tiled pieces of dE/da (the backward layers' A operands)
};
// FP32 B [N][K] (K contiguous) -> tiled pieces (pieces 1, 3: BF16; 2: the FP16
// pair of x scale); -1 on an unsupported shape
int launch_tile_operand(cudaStream_t st, int N, int K, int pieces, float scale, const float* src,
                        __nv_bfloat16* out);
// pieces: 1, 2 or 3 for every GEMM; 4: 3, the dE/dD GEMM 2
int fit_tc(cudaStream_t st, int64_t n, const int32_t* idx, const FitNetTC& net, int M, int m_lt,
           const float* T, float* dT, double* e_atom, const FitScratchTC& s, int pieces,
           int32_t* err);

// ---------------------------------------------------------------- MD / reductions
void launch_zero_forces(cudaStream_t st, int64_t n, unsigned long long* ffix);
void launch_force_finalize(cudaStream_t st, int64_t n, const unsigned long long* ffix, double* f,
                           int32_t* status);
// deterministic sums: out[k] = sum_i in[i*stride + k], k < width
void launch_sum_rows(cudaStream_t st, int64_t rows, int width, const double* in, double* part,
                     double* out);
int sum_rows_part_size(int64_t rows, int width);
// launch_sum_rows on nseg segments in one pass (seg_rows, seg_off: device
// arrays; out [nseg][width]); each segment's sum is bitwise the one
// launch_sum_rows gives on it alone
int64_t sum_rows_seg_part_size(int nseg, int width);
void launch_sum_rows_seg(cudaStream_t st, int nseg, const int64_t* seg_rows, const int64_t* seg_off,
                         int width, const double* in, double* part, double* out);
// out[c] = sum over r (in order, from 0) of in[r][c]; width <= 32
void launch_add_rows(cudaStream_t st, int nrows, int width, const double* in, double* out);
void launch_kick_drift(cudaStream_t st, int64_t n, double* x, double* v, const double* f,
                       const int32_t* types, const double* inv_mass_acc, double dt,
                       const double* xref, double half_skin2, int32_t* status);
void launch_kick(cudaStream_t st, int64_t n, double* v, const double* f, const int32_t* types,
                 const double* inv_mass_acc, const double* mass, double dt, double* ke_atom);
void launch_check_energy(cudaStream_t st, int64_t n, const double* e, int32_t* status);
void launch_map_types(cudaStream_t st, int64_t n, const int32_t* in, const int32_t* map, int nmap,
                      int32_t* out, int32_t* status);
