// C-ABI runtime: model loading, device buffers, neighbor-list management,
// the evaluation pipeline and velocity-Verlet MD.  All arithmetic of the
// method runs in the CUDA kernels; this file only sequences them.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <memory>
#include <mutex>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "dp_internal.h"

namespace {

constexpr double kAcc = 9.648533212e-3;  // (eV/A/amu) -> A/fs^2
constexpr double kKb = 8.617333262e-5;    // eV/K
constexpr double kEvA3Bar = 1.602176634e6;

// ------------------------------------------------------------------ fault injection
// DP_FAULT=alloc:N makes the N-th device allocation of the process fail
// (host-side injection; nothing on the GPU is disturbed).  DP_FAULT=wait:N
// gives the N-th launch of the tensor-core embedding forward a limit of zero
// polls on one bounded wait (its generator warps' wait for the MMAs to
// release a stage), so that wait runs out and the kernel takes its timeout
// path (DP_ERR_TIMEOUT); the waits that drain the CTA's own copies and MMAs
// keep the full limit.
std::atomic<long> g_alloc_count{0};  // allocations from several host threads
std::atomic<long> g_fwd_tc_count{0};
std::atomic<long> g_wait_fail_at{-1};
// bumped by every device (re)allocation: a captured CUDA graph holds raw
// pointers and is valid only while no buffer it uses has moved
std::atomic<unsigned long long> g_alloc_gen{0};
std::atomic<long> g_alloc_fail_at{-1};
std::once_flag g_fault_once;
// device bytes the library holds (every DevBuf), and the most it held since
// the last reset (dp_memory)
std::atomic<long long> g_dev_bytes{0};
std::atomic<long long> g_dev_peak{0};

void dev_bytes_add(long long b) {
  const long long now = g_dev_bytes.fetch_add(b) + b;
  long long pk = g_dev_peak.load();
  while (now > pk && !g_dev_peak.compare_exchange_weak(pk, now)) {
  }
}

void parse_fault() {
  std::call_once(g_fault_once, [] {
    const char* s = std::getenv("DP_FAULT");
    if (s && std::strncmp(s, "alloc:", 6) == 0) g_alloc_fail_at = std::atol(s + 6);
    if (s && std::strncmp(s, "wait:", 5) == 0) g_wait_fail_at = std::atol(s + 5);
  });
}

// the generator-wait limit of this launch of the tensor-core embedding
// forward: 0 for the injected launch, else -1 (the full limit)
long long fwd_tc_wait_limit() {
  parse_fault();
  const long k = ++g_fwd_tc_count;
  return (g_wait_fail_at > 0 && k == g_wait_fail_at) ? 0 : -1;
}

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes) {
    o.p = nullptr;
    o.bytes = 0;
  }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      if (p) {
        cudaFree(p);
        dev_bytes_add(-(long long)bytes);
      }
      p = o.p;
      bytes = o.bytes;
      o.p = nullptr;
      o.bytes = 0;
    }
    return *this;
  }
  ~DevBuf() {
    if (p) {
      cudaFree(p);
      dev_bytes_add(-(long long)bytes);
    }
  }
  void release() {
    if (p) {
      cudaFree(p);
      dev_bytes_add(-(long long)bytes);
    }
    p = nullptr;
    bytes = 0;
  }
};

cudaError_t ensure(DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (bytes <= b.bytes) return cudaSuccess;
  parse_fault();
  const long na = ++g_alloc_count;
  if (g_alloc_fail_at > 0 && na == g_alloc_fail_at) return cudaErrorMemoryAllocation;
  b.release();
  g_alloc_gen.fetch_add(1);
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e == cudaSuccess) {
    b.bytes = bytes;
    dev_bytes_add((long long)bytes);
  } else {
    b.p = nullptr;
    cudaGetLastError();  // clear the non-sticky allocation error
  }
  return e;
}

template <class T>
T* P(DevBuf& b) {
  return reinterpret_cast<T*>(b.p);
}

struct Work {
  int64_t n = 0;
  int cap = 0;
  double rlist = 0.0;
  CellGeom geom{};
  DevBuf x, xref, types, types_in, cellc, cell_count, cell_fill, cell_start, cell_tmp, cell_atoms,
      off, nlist, nn, T, dT, e_atom, ffix, f, vir_part, red_part, red_out, idx, ke, pairs;
  std::vector<int64_t> type_count, type_off;  // atoms per model type, offsets into idx
  bool have_idx = false;
  TileMap tiles{};  // the same grouping in tiles of 32 (tensor-core embedding)
  DevBuf tc_pairs, tc_hist, tc_range;  // sorted pairs / bin ends the forward leaves
  // several systems in one evaluation: tile index lists padded per system,
  // atom -> system, per-system first atom and cell edges, per-tile virial
  DevBuf bidx, sys_of, sys_base, sys_edge, vir_tile, vir_type, seg, seg_part, seg_out;
  size_t bytes() const {
    const DevBuf* all[] = {&x, &xref, &types, &types_in, &cellc, &cell_count, &cell_fill,
                           &cell_start, &cell_tmp, &cell_atoms, &off, &nlist, &nn, &T, &dT,
                           &e_atom, &ffix, &f, &vir_part, &red_part, &red_out, &idx, &ke, &pairs,
                           &tc_pairs, &tc_hist, &tc_range, &bidx, &sys_of, &sys_base, &sys_edge,
                           &vir_tile, &vir_type, &seg, &seg_part, &seg_out};
    size_t b = 0;
    for (const DevBuf* d : all) b += d->bytes;
    return b;
  }
};

// several independent systems in one atom array (host bookkeeping)
struct Batch {
  int nsys = 0;
  std::vector<int64_t> base;             // [nsys + 1] first atom of each system
  std::vector<std::array<double, 3>> L;  // box edges
  std::vector<double> boxes;             // [nsys][9] as given (state files)
  std::vector<CellGeom> geoms;           // cell grids of the last list build
  TileMap tm{};                          // tiles padded per system (index list in Work::bidx)
  // per system: (first tile, tiles) of each centre type present in it
  std::vector<std::vector<std::pair<int64_t, int64_t>>> sys_tiles;
  DevBuf geoms_dev;                      // CellGeom [nsys] for the batched mirror
};

}  // namespace

struct dp_handle {
  cudaStream_t st = nullptr;
  std::string err;
  bool dead = false;
  int ntypes_user = 0;
  int type_map[DP_MAXT] = {0};
  double rc = 0.0, rcs = 0.0;
  int sel[DP_MAXT] = {0};
  int Nm = 0;
  dp_options opt{};
  // model
  int ntypes = 0, n_emb = 0, emb_w[6] = {0}, M = 0, m_lt = 0, din = 0, n_fit = 0;
  int fit_w[DP_MAXFIT] = {0};
  DevBuf emb64, emb_off, table, fit32, sel_dev, map_dev, status;
  DevBuf tabF, tabB, tc_scratch;  // tensor-core embedding: tiled table pieces, per-CTA scratch
  DevBuf tanh_tab;                // Sec. 3.5 tanh table of the fitting net (tanh_table = 1)
  DevBuf pg, pg_fit_part, pg_tab_part;  // parameter gradients: FP64 result, FP32 partials
  // offsets (floats) of each type's W, W^T, b, w_out in fit32
  struct FitOfs {
    size_t W[DP_MAXFIT], WT[DP_MAXFIT], b[DP_MAXFIT], wout;
  };
  std::vector<FitOfs> fit_ofs;
  size_t fit_floats = 0;
  int n_int = 0;     // table intervals: n_fine of width h, then of width H
  int n_fine = 0;
  double h = 0.0, H = 0.0;
  FitNet nets[DP_MAXT];
  FitNetTC nets_tc[DP_MAXT];
  float b_out[DP_MAXT] = {0};
  DevBuf fitbuf, fit_bf16, fitbuf_tc, plain_w, plain_nets;
  FitScratch fs{};
  FitScratchTC fs_tc{};
  int32_t* status_host = nullptr;
  Work w;
  // profiling: event pairs recorded around each phase on the handle's stream
  bool prof = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev[DP_NPHASE];
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_pool;
  cudaStream_t cap_st = nullptr;  // private stream for CUDA-graph capture
  // the device buffers of the last destroyed system, reused by the next
  // dp_system_create (no cudaMalloc/cudaFree of the multi-GB lists per system)
  std::unique_ptr<Work> spare_work;
  DevBuf spare_v;
  ~dp_handle() {
    if (cap_st) cudaStreamDestroy(cap_st);
    for (auto& v : prof_ev)
      for (auto& e : v) prof_pool.push_back(e);
    for (auto& e : prof_pool) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
  }
};

struct dp_system {
  dp_handle* h = nullptr;
  Work w;
  std::unique_ptr<Batch> batch;  // several systems (dp_system_create_batch)
  DevBuf v, mass, inv_mass_acc, thermo;
  std::vector<int32_t> types_user;
  std::vector<double> mass_user;
  double box[9] = {0};
  int64_t step = 0;
  bool f_valid = false;
  // a step without a list rebuild, captured as one CUDA graph
  cudaGraphExec_t gexec = nullptr;
  unsigned long long ggen = 0;  // g_alloc_gen at capture
  double gdt = 0.0;
  unsigned long long glaunches = 0;  // kernel launches the graph replays
  int gplain = 0;  // plain steps since the last rebuild (lazy set-up done)
  bool gbroken = false;  // capture failed once: launch normally from now on
  ~dp_system() {
    if (gexec) cudaGraphExecDestroy(gexec);
  }
};

namespace {

// message of the last failed dp_create on this thread (dp_last_error(NULL))
thread_local std::string g_create_err;

dp_status fail(dp_handle* h, dp_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

dp_status cuda_fail(dp_handle* h, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return fail(h, DP_ERR_OOM, m);
  // errors from kernels (illegal address, launch failure, ...) poison the context
  if (e != cudaErrorInvalidValue && e != cudaErrorInvalidConfiguration) h->dead = true;
  return fail(h, DP_ERR_CUDA, m);
}

#define CK(call, where)                                 \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
  } while (0)

// Records a CUDA event pair around a phase when profiling is on.
struct Phase {
  dp_handle* h;
  int ph;
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  Phase(dp_handle* h_, int ph_) : h(h_), ph(ph_) {
    if (!h->prof) return;
    if (h->prof_pool.empty()) {
      cudaEvent_t a, b;
      if (cudaEventCreate(&a) != cudaSuccess) return;
      if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return;
      }
      h->prof_pool.push_back({a, b});
    }
    ev = h->prof_pool.back();
    h->prof_pool.pop_back();
    cudaEventRecord(ev.first, h->st);
  }
  void end() {
    if (!ev.first) return;
    cudaEventRecord(ev.second, h->st);
    h->prof_ev[ph].push_back(ev);
    ev.first = nullptr;
  }
  ~Phase() { end(); }
};

#define CKS(call)                          \
  do {                                     \
    dp_status s_ = (call);                 \
    if (s_ != DP_OK) return s_;            \
  } while (0)

// ------------------------------------------------------------------ model file
struct HostModel {
  int ntypes = 0, n_emb = 0, emb_w[6] = {0}, m_lt = 0, n_fit = 0, fit_w[DP_MAXFIT] = {0};
  std::vector<double> data;
  std::vector<int64_t> emb_off;   // per (pair, layer): offset of W in data
  std::vector<int64_t> fit_off;   // per (type, layer): offset of W; then w_out, b_out
};

bool read_model(const char* path, HostModel& m, std::string& why) {
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    why = std::string("cannot open model file ") + path;
    return false;
  }
  auto rd = [&](void* p, size_t sz, size_t cnt) { return std::fread(p, sz, cnt, f) == cnt; };
  char magic[8];
  int32_t v[2];
  bool ok = rd(magic, 1, 8) && std::memcmp(magic, "DPSEAV01", 8) == 0 && rd(v, 4, 2);
  int nint = 2;
  if (ok) {
    m.ntypes = v[0];
    m.n_emb = v[1];
    ok = m.ntypes >= 1 && m.ntypes <= DP_MAXT && m.n_emb >= 1 && m.n_emb <= 6;
  }
  if (ok) ok = rd(m.emb_w, 4, m.n_emb) && rd(v, 4, 2);
  if (ok) {
    nint += m.n_emb + 2;
    m.m_lt = v[0];
    m.n_fit = v[1];
    ok = m.n_fit >= 1 && m.n_fit <= DP_MAXFIT;
  }
  if (ok) {
    ok = rd(m.fit_w, 4, m.n_fit);
    nint += m.n_fit;
  }
  if (ok && nint % 2) ok = rd(v, 4, 1);
  if (ok)
    for (int k = 1; k < m.n_emb; ++k) ok = ok && m.emb_w[k] == 2 * m.emb_w[k - 1];
  const int M = ok ? m.emb_w[m.n_emb - 1] : 0;
  if (ok) ok = m.m_lt >= 1 && m.m_lt <= M;
  if (!ok) {
    std::fclose(f);
    why = "malformed model header";
    return false;
  }
  const int din = M * m.m_lt;
  int64_t tot = 0;
  const int np = m.ntypes * m.ntypes;
  for (int p = 0; p < np; ++p) {
    int prev = 1;
    for (int k = 0; k < m.n_emb; ++k) {
      m.emb_off.push_back(tot);
      tot += (int64_t)prev * m.emb_w[k] + m.emb_w[k];
      prev = m.emb_w[k];
    }
  }
  for (int t = 0; t < m.ntypes; ++t) {
    int prev = din;
    for (int k = 0; k < m.n_fit; ++k) {
      m.fit_off.push_back(tot);
      tot += (int64_t)prev * m.fit_w[k] + m.fit_w[k];
      prev = m.fit_w[k];
    }
    m.fit_off.push_back(tot);  // w_out then b_out
    tot += prev + 1;
  }
  m.data.resize(tot);
  ok = rd(m.data.data(), sizeof(double), (size_t)tot);
  char extra;
  if (ok && std::fread(&extra, 1, 1, f) != 0) ok = false;
  std::fclose(f);
  if (!ok) why = "model file size does not match its header";
  return ok;
}

// ------------------------------------------------------------------ helpers
dp_status box_lengths(dp_handle* h, const double* box, double* L) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      if (a != b && box[a * 3 + b] != 0.0)
        return fail(h, DP_ERR_BOX, "only orthorhombic boxes are supported");
  for (int a = 0; a < 3; ++a) {
    L[a] = box[a * 4];
    if (!(L[a] > 0.0) || !std::isfinite(L[a])) return fail(h, DP_ERR_BOX, "box edge must be > 0");
  }
  return DP_OK;
}

EnvParams env_params(const dp_handle* h) {
  EnvParams ep{};
  ep.rc2 = (float)(h->rc * h->rc);
  ep.rc = (float)h->rc;
  ep.rcs = (float)h->rcs;
  ep.inv_w = (float)(1.0 / (h->rc - h->rcs));
  ep.inv_h = (float)(1.0 / h->h);
  ep.h = (float)h->h;
  ep.s_fine = (float)(h->n_fine * h->h);
  ep.inv_H = (float)(1.0 / h->H);
  ep.smax = (float)(h->n_fine * h->h + (h->n_int - h->n_fine) * h->H);
  ep.inv_nm = (float)(1.0 / h->Nm);
  ep.n_int = h->n_int;
  ep.n_fine = h->n_fine;
  ep.M = h->M;
  ep.ntypes = h->ntypes;
  return ep;
}

dp_status read_status(dp_handle* h) {
  CK(cudaMemcpyAsync(h->status_host, P<int32_t>(h->status), sizeof(int32_t) * ST_NWORDS,
                     cudaMemcpyDeviceToHost, h->st),
     "status copy");
  CK(cudaStreamSynchronize(h->st), "device execution");
  return DP_OK;
}

dp_status clear_status(dp_handle* h) {
  CK(cudaMemsetAsync(h->status.p, 0, sizeof(int32_t) * ST_NWORDS, h->st), "status clear");
  return DP_OK;
}

dp_status status_errors(dp_handle* h) {
  const int32_t* s = h->status_host;
  char buf[160];
  if (s[ST_BADTYPE]) {
    std::snprintf(buf, sizeof buf, "%d atoms have a type outside [0, %d)", s[ST_BADTYPE],
                  h->ntypes_user);
    return fail(h, DP_ERR_ARG, buf);
  }
  if (s[ST_SEL]) {
    std::snprintf(buf, sizeof buf, "%d atoms have more neighbors of a type within rc than sel",
                  s[ST_SEL]);
    return fail(h, DP_ERR_SEL_OVERFLOW, buf);
  }
  if (s[ST_SKIN]) {
    std::snprintf(buf, sizeof buf, "%d atoms moved more than skin/2 between rebuilds", s[ST_SKIN]);
    return fail(h, DP_ERR_SKIN, buf);
  }
  if (s[ST_RANGE]) {
    std::snprintf(buf, sizeof buf, "%d pairs have s outside the table domain [0, %g]", s[ST_RANGE],
                  h->n_fine * h->h + (h->n_int - h->n_fine) * h->H);
    return fail(h, DP_ERR_TABLE_RANGE, buf);
  }
  if (s[ST_TIMEOUT]) {
    std::snprintf(buf, sizeof buf, "%d bounded device waits gave up", s[ST_TIMEOUT]);
    return fail(h, DP_ERR_TIMEOUT, buf);
  }
  if (s[ST_NONFINITE]) {
    std::snprintf(buf, sizeof buf, "%d non-finite energies or pair forces", s[ST_NONFINITE]);
    return fail(h, DP_ERR_NONFINITE, buf);
  }
  return DP_OK;
}

// per-atom buffers of a work area
dp_status ensure_atoms(dp_handle* h, Work& w, int64_t n) {
  const size_t N = (size_t)std::max<int64_t>(n, 1);
  CK(ensure(w.x, N * 3 * sizeof(double)), "alloc x");
  CK(ensure(w.xref, N * 3 * sizeof(double)), "alloc xref");
  CK(ensure(w.types, N * sizeof(int32_t)), "alloc types");
  CK(ensure(w.types_in, N * sizeof(int32_t)), "alloc types");
  CK(ensure(w.cellc, N * sizeof(int32_t)), "alloc cells");
  CK(ensure(w.cell_tmp, N * sizeof(int32_t)), "alloc cells");
  CK(ensure(w.cell_atoms, N * sizeof(int32_t)), "alloc cells");
  CK(ensure(w.off, N * sizeof(float4)), "alloc offsets");
  CK(ensure(w.nn, N * sizeof(int32_t)), "alloc nn");
  CK(ensure(w.T, N * 4 * h->M * sizeof(float)), "alloc T");
  CK(ensure(w.dT, N * 4 * h->M * sizeof(float)), "alloc dT");
  CK(ensure(w.e_atom, N * sizeof(double)), "alloc e");
  CK(ensure(w.ke, N * sizeof(double)), "alloc ke");
  CK(ensure(w.ffix, N * 3 * sizeof(unsigned long long)), "alloc f");
  CK(ensure(w.f, N * 3 * sizeof(double)), "alloc f");
  CK(ensure(w.idx, N * sizeof(int32_t)), "alloc idx");
  CK(ensure(w.vir_part,
            (size_t)std::max<int64_t>(std::max(tab_kernel_slots(n), plain_kernel_slots(n)),
                                      tab_tc_slots()) *
                9 * sizeof(double)),
     "alloc virial");
  CK(ensure(w.red_part, (size_t)sum_rows_part_size(n, 9) * sizeof(double)), "alloc red");
  CK(ensure(w.red_out, 32 * sizeof(double)), "alloc red");
  CK(ensure(w.pairs, sizeof(unsigned long long)), "alloc counters");
  w.n = n;
  return DP_OK;
}

// per-type index lists for the fitting stage (stable: ascending atom index)
dp_status set_types(dp_handle* h, Work& w, const int32_t* types_user_host) {
  const int64_t n = w.n;
  w.type_count.assign(h->ntypes, 0);
  w.type_off.assign(h->ntypes + 1, 0);
  std::vector<int32_t> mt(n);
  for (int64_t i = 0; i < n; ++i) {
    int t = types_user_host[i];
    if (t < 0 || t >= h->ntypes_user) return fail(h, DP_ERR_ARG, "atom type out of range");
    mt[i] = h->type_map[t];
    w.type_count[mt[i]]++;
  }
  for (int t = 0; t < h->ntypes; ++t) w.type_off[t + 1] = w.type_off[t] + w.type_count[t];
  w.have_idx = h->ntypes > 1;
  w.tiles = TileMap{};
  w.tiles.ntypes = h->ntypes;
  for (int t = 0; t < h->ntypes; ++t) {
    w.tiles.atom_off[t] = w.type_off[t];
    w.tiles.atom_cnt[t] = w.type_count[t];
    w.tiles.tile_off[t + 1] = w.tiles.tile_off[t] + (w.type_count[t] + 31) / 32;
  }
  w.tiles.idx = w.have_idx ? P<int32_t>(w.idx) : nullptr;
  if (h->opt.tabulated && h->opt.embed_precision == 2) {
    const EnvParams ep = env_params(h);
    const int64_t ntile = w.tiles.tile_off[h->ntypes];
    CK(ensure(w.tc_pairs, (size_t)std::max<int64_t>(tab_tc_pair_elems(ep, ntile), 1) * 16),
       "alloc sorted pairs");
    CK(ensure(w.tc_hist, (size_t)std::max<int64_t>(tab_tc_hist_elems(ep, ntile), 8) * 2),
       "alloc bin ends");
    CK(ensure(w.tc_range, (size_t)std::max<int64_t>(ntile, 1) * 8), "alloc bin ranges");
    CK(ensure(w.vir_tile, (size_t)std::max<int64_t>(ntile, 1) * 9 * sizeof(double)), "alloc virial");
    CK(ensure(w.vir_type, DP_MAXT * 9 * sizeof(double)), "alloc virial");
  }
  if (n > 0) {
    CK(cudaMemcpyAsync(w.types.p, mt.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, h->st),
       "types upload");
    if (w.have_idx) {
      std::vector<int32_t> idx(n);
      std::vector<int64_t> fill(w.type_off.begin(), w.type_off.end() - 1);
      for (int64_t i = 0; i < n; ++i) idx[fill[mt[i]]++] = (int32_t)i;
      CK(cudaMemcpyAsync(w.idx.p, idx.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, h->st),
         "idx upload");
    }
    CK(cudaStreamSynchronize(h->st), "types upload");
  }
  return DP_OK;
}

dp_status ensure_fit_scratch(dp_handle* h, int64_t rows_needed) {
  int64_t rows = std::min<int64_t>(std::max<int64_t>(rows_needed, 1), 131072);
  if (rows <= h->fs.rows) return DP_OK;
  int wmax = 0;
  for (int k = 0; k < h->n_fit; ++k) wmax = std::max(wmax, h->fit_w[k]);
  size_t per = 2 * (size_t)h->din + 3 * (size_t)wmax;
  for (int k = 0; k < h->n_fit; ++k) per += 2 * (size_t)h->fit_w[k];
  CK(ensure(h->fitbuf, per * rows * sizeof(float)), "alloc fitting scratch");
  float* q = P<float>(h->fitbuf);
  FitScratch& s = h->fs;
  s.rows = rows;
  s.D = q;
  q += rows * h->din;
  s.dD = q;
  q += rows * h->din;
  for (int k = 0; k < h->n_fit; ++k) {
    s.t[k] = q;
    q += rows * h->fit_w[k];
    s.z[k] = q;
    q += rows * h->fit_w[k];
  }
  s.gz = q;
  q += rows * wmax;
  s.gp = q;
  q += rows * wmax;
  s.gz2 = q;
  return DP_OK;
}

// Wrap positions, bin them into cells of edge >= rlist, sort the cells and
// build the lists (growing the capacity until every list fits).
dp_status rebuild(dp_handle* h, Work& w, const double* L, double rlist) {
  CellGeom g{};
  long long ncell = 1;
  for (int a = 0; a < 3; ++a) {
    if (L[a] < rlist)
      return fail(h, DP_ERR_BOX, "a box edge is shorter than the neighbor-list cutoff");
    g.L[a] = L[a];
    g.nc[a] = std::max(1, (int)std::floor(L[a] / rlist));
    g.edge[a] = L[a] / g.nc[a];
    g.edgef[a] = (float)g.edge[a];
    ncell *= g.nc[a];
  }
  if (ncell > (1LL << 30)) return fail(h, DP_ERR_BOX, "too many cells");
  g.ncell = ncell;
  w.geom = g;
  w.rlist = rlist;
  const int64_t n = w.n;
  if (n == 0) return DP_OK;
  Phase ph(h, 0);
  CK(ensure(w.cell_count, (ncell + 1) * sizeof(int32_t)), "alloc cells");
  CK(ensure(w.cell_fill, (ncell + 1) * sizeof(int32_t)), "alloc cells");
  CK(ensure(w.cell_start, (ncell + 1) * sizeof(int32_t)), "alloc cells");
  CK(cudaMemsetAsync(w.cell_count.p, 0, (ncell + 1) * sizeof(int32_t), h->st), "memset");
  CK(cudaMemsetAsync(w.cell_fill.p, 0, (ncell + 1) * sizeof(int32_t), h->st), "memset");
  launch_wrap_bin(h->st, n, P<double>(w.x), g, P<int32_t>(w.cellc), P<int32_t>(w.cell_count));
  launch_scan(h->st, P<int32_t>(w.cell_count), P<int32_t>(w.cell_start), ncell);
  launch_scatter(h->st, n, P<int32_t>(w.cellc), P<int32_t>(w.cell_start), P<int32_t>(w.cell_fill),
                 P<int32_t>(w.cell_tmp));
  launch_cell_sort(h->st, ncell, P<int32_t>(w.cell_start), P<int32_t>(w.cell_tmp),
                   P<int32_t>(w.cell_atoms));
  launch_mirror(h->st, n, P<double>(w.x), P<int32_t>(w.cellc), P<int32_t>(w.types), g,
                P<float4>(w.off));
  CK(cudaMemcpyAsync(w.xref.p, w.x.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, h->st),
     "xref");
  if (w.cap == 0) {
    const double vol = L[0] * L[1] * L[2];
    const double est = (double)n / vol * 4.18879020479 * rlist * rlist * rlist;
    w.cap = std::max(32, ((int)(1.25 * est + 32) + 31) / 32 * 32);
  }
  const float rc2 = (float)(h->rc * h->rc);
  for (int attempt = 0; attempt < 3; ++attempt) {
    CK(ensure(w.nlist, (size_t)n * w.cap * sizeof(uint32_t)), "alloc neighbor list");
    CK(cudaMemsetAsync(P<int32_t>(h->status) + ST_MAXLIST, 0, 2 * sizeof(int32_t), h->st), "memset");
    launch_build_list(h->st, n, P<double>(w.x), P<int32_t>(w.cellc), P<float4>(w.off),
                      P<int32_t>(w.cell_start), P<int32_t>(w.cell_atoms), g, rlist, rc2,
                      h->ntypes, P<int32_t>(h->sel_dev), w.cap, P<uint32_t>(w.nlist),
                      P<int32_t>(w.nn), P<int32_t>(h->status));
    CK(cudaGetLastError(), "neighbor kernels");
    CKS(read_status(h));
    if (h->status_host[ST_LISTOVF] == 0) return DP_OK;
    w.cap = ((int)(h->status_host[ST_MAXLIST] * 1.1) + 8 + 31) / 32 * 32;
  }
  return fail(h, DP_ERR_CUDA, "neighbor list capacity did not converge");
}

// neighbor lists of several systems (atoms [base[s], base[s+1]) in a box of
// edges L[s]) into one list array: each system is binned and listed on its
// own (the cell arrays are reused in stream order); entries hold
// system-local indices
dp_status rebuild_batch(dp_handle* h, Work& w, const std::vector<int64_t>& base,
                        const std::vector<std::array<double, 3>>& Ls, double rlist,
                        std::vector<CellGeom>& gs) {
  const int nsys = (int)base.size() - 1;
  const int64_t n = w.n;
  gs.assign(nsys, CellGeom{});
  long long maxcell = 1;
  double est = 0.0;
  for (int q = 0; q < nsys; ++q) {
    CellGeom g{};
    long long ncell = 1;
    for (int a = 0; a < 3; ++a) {
      if (Ls[q][a] < rlist)
        return fail(h, DP_ERR_BOX, "a box edge is shorter than the neighbor-list cutoff");
      g.L[a] = Ls[q][a];
      g.nc[a] = std::max(1, (int)std::floor(Ls[q][a] / rlist));
      g.edge[a] = Ls[q][a] / g.nc[a];
      g.edgef[a] = (float)g.edge[a];
      ncell *= g.nc[a];
    }
    if (ncell > (1LL << 30)) return fail(h, DP_ERR_BOX, "too many cells");
    g.ncell = ncell;
    gs[q] = g;
    maxcell = std::max(maxcell, ncell);
    const double vol = Ls[q][0] * Ls[q][1] * Ls[q][2];
    est = std::max(est, (double)(base[q + 1] - base[q]) / vol * 4.18879020479 * rlist * rlist * rlist);
  }
  w.geom = gs.empty() ? CellGeom{} : gs[0];
  w.rlist = rlist;
  if (n == 0) return DP_OK;
  CK(ensure(w.cell_count, (maxcell + 1) * sizeof(int32_t)), "alloc cells");
  CK(ensure(w.cell_fill, (maxcell + 1) * sizeof(int32_t)), "alloc cells");
  CK(ensure(w.cell_start, (maxcell + 1) * sizeof(int32_t)), "alloc cells");
  w.cap = std::max(32, ((int)(1.25 * est + 32) + 31) / 32 * 32);
  const float rc2 = (float)(h->rc * h->rc);
  for (int attempt = 0; attempt < 3; ++attempt) {
    CK(ensure(w.nlist, (size_t)n * w.cap * sizeof(uint32_t)), "alloc neighbor list");
    CK(cudaMemsetAsync(P<int32_t>(h->status) + ST_MAXLIST, 0, 2 * sizeof(int32_t), h->st), "memset");
    for (int q = 0; q < nsys; ++q) {
      const int64_t b = base[q], ns = base[q + 1] - base[q];
      if (ns == 0) continue;
      const CellGeom& g = gs[q];
      CK(cudaMemsetAsync(w.cell_count.p, 0, (g.ncell + 1) * sizeof(int32_t), h->st), "memset");
      CK(cudaMemsetAsync(w.cell_fill.p, 0, (g.ncell + 1) * sizeof(int32_t), h->st), "memset");
      double* xb = P<double>(w.x) + 3 * b;
      int32_t* cb = P<int32_t>(w.cellc) + b;
      float4* ob = P<float4>(w.off) + b;
      launch_wrap_bin(h->st, ns, xb, g, cb, P<int32_t>(w.cell_count));
      launch_scan(h->st, P<int32_t>(w.cell_count), P<int32_t>(w.cell_start), g.ncell);
      launch_scatter(h->st, ns, cb, P<int32_t>(w.cell_start), P<int32_t>(w.cell_fill),
                     P<int32_t>(w.cell_tmp));
      launch_cell_sort(h->st, g.ncell, P<int32_t>(w.cell_start), P<int32_t>(w.cell_tmp),
                       P<int32_t>(w.cell_atoms));
      launch_mirror(h->st, ns, xb, cb, P<int32_t>(w.types) + b, g, ob);
      launch_build_list(h->st, ns, xb, cb, ob, P<int32_t>(w.cell_start), P<int32_t>(w.cell_atoms),
                        g, rlist, rc2, h->ntypes, P<int32_t>(h->sel_dev), w.cap,
                        P<uint32_t>(w.nlist) + (size_t)b * w.cap, P<int32_t>(w.nn) + b,
                        P<int32_t>(h->status));
    }
    CK(cudaGetLastError(), "neighbor kernels");
    CKS(read_status(h));
    if (h->status_host[ST_LISTOVF] == 0) return DP_OK;
    w.cap = ((int)(h->status_host[ST_MAXLIST] * 1.1) + 8 + 31) / 32 * 32;
  }
  return fail(h, DP_ERR_CUDA, "neighbor list capacity did not converge");
}

// 16-bit pieces per fitting operand of each fit_precision: 1 one BF16 piece,
// 2 three BF16 pieces (FP32-accurate), 3 the FP16 pair (near-FP32), 4 three
// BF16 pieces with the dE/dD GEMM's operands an FP16 pair (fit_tc's code 4)
static int fit_pieces(int fit_precision) {
  return fit_precision == 2 ? 3 : fit_precision == 3 ? 2 : fit_precision == 4 ? 4 : 1;
}

dp_status ensure_fit_scratch_tc(dp_handle* h, int64_t rows_needed) {
  const int PCN = 3;  // room for three pieces serves every tensor-core mode
  // chunks of 32 x 152 tiles of 128 rows (whole waves on 152 SMs; 8 and 16
  // waves measured 1.6 and 0.55 ms slower per 4M-atom evaluation: more
  // launches, each with its pipeline fill and a last tile whose epilogue
  // nothing overlaps)
  int64_t rows = std::min<int64_t>(std::max<int64_t>(rows_needed, 1), 32 * 152 * 128);
  rows = (rows + 127) / 128 * 128;
  if (rows <= h->fs_tc.rows) return DP_OK;
  int wmax = 0;
  for (int k = 0; k < h->n_fit; ++k) wmax = std::max(wmax, h->fit_w[k]);
  size_t bytes = rows * (size_t)wmax * (4 + 3 * 2 * PCN);
  for (int k = 0; k < h->n_fit; ++k) bytes += rows * (size_t)h->fit_w[k] * (4 + 4);
  bytes += 64 * 256;
  CK(ensure(h->fitbuf_tc, bytes), "alloc tensor-core fitting scratch");
  unsigned char* q = P<unsigned char>(h->fitbuf_tc);
  auto take = [&](size_t b) {
    unsigned char* p = q;
    q += (b + 255) / 256 * 256;
    return p;
  };
  FitScratchTC& s = h->fs_tc;
  s.rows = rows;
  s.wmax = wmax;
  for (int k = 0; k < h->n_fit; ++k) {
    s.t[k] = (float*)take(rows * h->fit_w[k] * 4);
    s.z[k] = (float*)take(rows * h->fit_w[k] * 4);
  }
  s.gz = (float*)take(rows * wmax * 4);
  s.zh = (__nv_bfloat16*)take(rows * wmax * 2 * PCN);
  s.gph[0] = (__nv_bfloat16*)take(rows * wmax * 2 * PCN);
  s.gph[1] = (__nv_bfloat16*)take(rows * wmax * 2 * PCN);
  return DP_OK;
}

// fitting stage of one centre type: E_i and dE/dT for cnt atoms (idx or all)
dp_status run_fitting(dp_handle* h, int t, int64_t cnt, const int32_t* idx, const float* T,
                      float* dT, double* e_atom) {
  if (h->opt.fit_precision >= 1) {
    CKS(ensure_fit_scratch_tc(h, cnt));
    if (fit_tc(h->st, cnt, idx, h->nets_tc[t], h->M, h->m_lt, T, dT, e_atom, h->fs_tc,
               fit_pieces(h->opt.fit_precision), P<int32_t>(h->status) + ST_TIMEOUT))
      return fail(h, DP_ERR_UNIMPLEMENTED, "tensor-core fitting cannot run this model shape");
    return DP_OK;
  }
  CKS(ensure_fit_scratch(h, cnt));
  if (fit_simt(h->st, cnt, idx, h->nets[t], h->M, h->m_lt, T, dT, e_atom, h->fs))
    return fail(h, DP_ERR_CUDA, "fitting kernels failed to launch");
  return DP_OK;
}

// environment matrix + embedding + contraction: T of every atom
dp_status embed_forward(dp_handle* h, Work& w, const EnvParams& ep) {
  if (h->opt.tabulated && h->opt.embed_precision == 2) {
    if (launch_tab_fwd_tc(h->st, w.tiles, P<float4>(w.off), P<uint32_t>(w.nlist),
                          P<int32_t>(w.nn), w.cap, w.geom, ep, P<__nv_bfloat16>(h->tabF),
                          P<float>(h->tc_scratch), P<float4>(w.tc_pairs), P<uint16_t>(w.tc_hist),
                          P<int2>(w.tc_range), P<float>(w.T), P<int32_t>(h->status),
                          P<unsigned long long>(w.pairs), nullptr, nullptr, nullptr,
                          fwd_tc_wait_limit()))
      return fail(h, DP_ERR_UNIMPLEMENTED, "tensor-core embedding cannot run this model shape");
  } else if (h->opt.tabulated) {
    if (launch_tab_fwd(h->st, w.n, P<float4>(w.off), P<uint32_t>(w.nlist), P<int32_t>(w.nn),
                       w.cap, w.geom, ep, P<float>(h->table), P<float>(w.T),
                       P<int32_t>(h->status), P<unsigned long long>(w.pairs)))
      return fail(h, DP_ERR_UNIMPLEMENTED, "tabulated kernel cannot run this model shape");
  } else {
    if (launch_plain_fwd(h->st, w.n, P<float4>(w.off), P<uint32_t>(w.nlist), P<int32_t>(w.nn),
                         w.cap, w.geom, ep, h->plain_nets.p, h->emb_w[0], P<float>(w.T),
                         P<unsigned long long>(w.pairs)))
      return fail(h, DP_ERR_UNIMPLEMENTED, "plain kernel cannot run this model shape");
  }
  return DP_OK;
}

// energy, forces, virial from the current list and offsets
dp_status evaluate(dp_handle* h, Work& w) {
  const int64_t n = w.n;
  if (n == 0) {
    CK(cudaMemsetAsync(w.red_out.p, 0, 16 * sizeof(double), h->st), "memset");
    return DP_OK;
  }
  const EnvParams ep = env_params(h);
  launch_zero_forces(h->st, n, P<unsigned long long>(w.ffix));
  CK(cudaMemsetAsync(w.pairs.p, 0, sizeof(unsigned long long), h->st), "memset");
  {
    Phase ph(h, 1);
    CKS(embed_forward(h, w, ep));
  }
  Phase ph_fit(h, 2);
  for (int t = 0; t < h->ntypes; ++t) {
    const int64_t cnt = w.have_idx ? w.type_count[t] : n;
    if (cnt == 0) continue;
    const int32_t* idx = w.have_idx ? P<int32_t>(w.idx) + w.type_off[t] : nullptr;
    CKS(run_fitting(h, t, cnt, idx, P<float>(w.T), P<float>(w.dT), P<double>(w.e_atom)));
    if (!w.have_idx) break;
  }
  ph_fit.end();
  {
    Phase ph(h, 3);
    if (h->opt.tabulated && h->opt.embed_precision == 2) {
      if (launch_tab_bwd_tc(h->st, w.tiles, P<float4>(w.tc_pairs), P<uint16_t>(w.tc_hist),
                            P<int2>(w.tc_range), ep, P<__nv_bfloat16>(h->tabB), P<float>(w.dT),
                            P<unsigned long long>(w.ffix), P<double>(w.vir_part),
                            (int)tab_tc_slots(), P<int32_t>(h->status), P<double>(w.vir_tile)))
        return fail(h, DP_ERR_UNIMPLEMENTED, "tensor-core embedding cannot run this model shape");
    } else if (h->opt.tabulated) {
      if (launch_tab_bwd(h->st, n, P<float4>(w.off), P<uint32_t>(w.nlist), P<int32_t>(w.nn),
                         w.cap, w.geom, ep, P<float>(h->table), P<float>(w.dT),
                         P<unsigned long long>(w.ffix), P<double>(w.vir_part),
                         tab_kernel_slots(n), P<int32_t>(h->status)))
        return fail(h, DP_ERR_UNIMPLEMENTED, "tabulated kernel cannot run this model shape");
    } else {
      CK(cudaMemsetAsync(w.vir_part.p, 0, w.vir_part.bytes, h->st), "memset");
      if (launch_plain_bwd(h->st, n, P<float4>(w.off), P<uint32_t>(w.nlist), P<int32_t>(w.nn),
                           w.cap, w.geom, ep, h->plain_nets.p, h->emb_w[0], P<float>(w.dT),
                           P<unsigned long long>(w.ffix), P<double>(w.vir_part),
                           plain_kernel_slots(n), P<int32_t>(h->status)))
        return fail(h, DP_ERR_UNIMPLEMENTED, "plain kernel cannot run this model shape");
    }
  }
  Phase ph_int(h, 4);
  launch_force_finalize(h->st, n, P<unsigned long long>(w.ffix), P<double>(w.f),
                        P<int32_t>(h->status));
  launch_sum_rows(h->st, n, 1, P<double>(w.e_atom), P<double>(w.red_part), P<double>(w.red_out));
  if (h->opt.tabulated && h->opt.embed_precision == 2) {
    // the virial from one row per tile: summed per centre type, the types
    // then added in order (the same sums dp_compute_batch makes per system)
    int k = 0;
    for (int t = 0; t < h->ntypes; ++t) {
      const int64_t nt = w.tiles.tile_off[t + 1] - w.tiles.tile_off[t];
      if (nt == 0) continue;
      launch_sum_rows(h->st, nt, 9, P<double>(w.vir_tile) + w.tiles.tile_off[t] * 9,
                      P<double>(w.red_part), P<double>(w.vir_type) + 9 * k);
      ++k;
    }
    launch_add_rows(h->st, k, 9, P<double>(w.vir_type), P<double>(w.red_out) + 1);
  } else {
    const int64_t vslots = !h->opt.tabulated ? plain_kernel_slots(n) : tab_kernel_slots(n);
    launch_sum_rows(h->st, vslots, 9,
                    P<double>(w.vir_part), P<double>(w.red_part), P<double>(w.red_out) + 1);
  }
  launch_check_energy(h->st, n, P<double>(w.e_atom), P<int32_t>(h->status));
  CK(cudaGetLastError(), "evaluation kernels");
  return DP_OK;
}

// ------------------------------------------------------------------ several systems
dp_status batch_init(dp_handle* h, Batch& b, int nsys, const int64_t* natoms,
                     const double* boxes) {
  if (nsys < 0 || (nsys > 0 && (!natoms || !boxes))) return fail(h, DP_ERR_ARG, "bad argument");
  if (!(h->opt.tabulated && h->opt.embed_precision == 2))
    return fail(h, DP_ERR_UNIMPLEMENTED,
                "several systems at once need the tabulated tensor-core embedding "
                "(embed_precision 2)");
  b.nsys = nsys;
  b.base.assign(nsys + 1, 0);
  for (int q = 0; q < nsys; ++q) {
    if (natoms[q] < 0) return fail(h, DP_ERR_ARG, "negative atom count");
    b.base[q + 1] = b.base[q] + natoms[q];
  }
  if (b.base[nsys] >= (1LL << 27)) return fail(h, DP_ERR_ARG, "at most 2^27 atoms per call");
  b.L.assign(nsys, {0.0, 0.0, 0.0});
  for (int q = 0; q < nsys; ++q) CKS(box_lengths(h, boxes + 9 * q, b.L[q].data()));
  b.boxes.assign(boxes, boxes + 9 * (size_t)nsys);
  return DP_OK;
}

// tiles of 32 padded per system (a tile belongs to one system, its virial row
// to that system) and the atom -> system tables; after load_coords
dp_status batch_tiles(dp_handle* h, Work& w, Batch& b, const int32_t* types_user) {
  const int nsys = b.nsys;
  const int64_t n = b.base[nsys];
  std::vector<int32_t> pidx;
  b.sys_tiles.assign(nsys, {});
  TileMap tm{};
  tm.ntypes = h->ntypes;
  for (int t = 0; t < h->ntypes; ++t) {
    tm.atom_off[t] = (int64_t)pidx.size();
    tm.tile_off[t] = (int64_t)pidx.size() / 32;
    for (int q = 0; q < nsys; ++q) {
      const int64_t t0 = (int64_t)pidx.size() / 32;
      for (int64_t i = b.base[q]; i < b.base[q + 1]; ++i)
        if (h->type_map[types_user[i]] == t) pidx.push_back((int32_t)i);
      while (pidx.size() % 32) pidx.push_back(-1);
      const int64_t t1 = (int64_t)pidx.size() / 32;
      if (t1 > t0) b.sys_tiles[q].push_back({t0, t1 - t0});
    }
    tm.atom_cnt[t] = (int64_t)pidx.size() - tm.atom_off[t];
  }
  tm.tile_off[h->ntypes] = (int64_t)pidx.size() / 32;
  const int64_t ntile = tm.tile_off[h->ntypes];
  std::vector<int32_t> sys_of(std::max<int64_t>(n, 1), 0), sys_base(std::max(nsys, 1), 0);
  for (int q = 0; q < nsys; ++q) {
    for (int64_t i = b.base[q]; i < b.base[q + 1]; ++i) sys_of[i] = q;
    sys_base[q] = (int32_t)b.base[q];
  }
  const EnvParams ep = env_params(h);
  CK(ensure(w.bidx, std::max<size_t>(pidx.size(), 1) * sizeof(int32_t)), "alloc tiles");
  CK(ensure(w.sys_of, sys_of.size() * sizeof(int32_t)), "alloc systems");
  CK(ensure(w.sys_base, sys_base.size() * sizeof(int32_t)), "alloc systems");
  CK(ensure(w.sys_edge, (size_t)std::max(nsys, 1) * sizeof(float4)), "alloc systems");
  CK(ensure(b.geoms_dev, (size_t)std::max(nsys, 1) * sizeof(CellGeom)), "alloc systems");
  CK(ensure(w.vir_tile, (size_t)std::max<int64_t>(ntile, 1) * 9 * sizeof(double)), "alloc virial");
  CK(ensure(w.tc_pairs, (size_t)std::max<int64_t>(tab_tc_pair_elems(ep, ntile), 1) * 16),
     "alloc sorted pairs");
  CK(ensure(w.tc_hist, (size_t)std::max<int64_t>(tab_tc_hist_elems(ep, ntile), 8) * 2),
     "alloc bin ends");
  CK(ensure(w.tc_range, (size_t)std::max<int64_t>(ntile, 1) * 8), "alloc bin ranges");
  if (!pidx.empty())
    CK(cudaMemcpyAsync(w.bidx.p, pidx.data(), pidx.size() * sizeof(int32_t),
                       cudaMemcpyHostToDevice, h->st),
       "tiles upload");
  CK(cudaMemcpyAsync(w.sys_of.p, sys_of.data(), sys_of.size() * sizeof(int32_t),
                     cudaMemcpyHostToDevice, h->st),
     "systems upload");
  CK(cudaMemcpyAsync(w.sys_base.p, sys_base.data(), sys_base.size() * sizeof(int32_t),
                     cudaMemcpyHostToDevice, h->st),
     "systems upload");
  // the host vectors are freed on return: wait for the copies
  CK(cudaStreamSynchronize(h->st), "systems upload");
  tm.idx = P<int32_t>(w.bidx);
  b.tm = tm;
  return DP_OK;
}

// the systems' neighbor lists and, for the kernels, their cell grids and edges
dp_status batch_rebuild(dp_handle* h, Work& w, Batch& b, double rlist) {
  CKS(rebuild_batch(h, w, b.base, b.L, rlist, b.geoms));
  const int nsys = b.nsys;
  if (nsys == 0 || w.n == 0) return DP_OK;
  std::vector<float4> edge(nsys);
  for (int q = 0; q < nsys; ++q)
    edge[q] = make_float4(b.geoms[q].edgef[0], b.geoms[q].edgef[1], b.geoms[q].edgef[2], 0.0f);
  CK(cudaMemcpyAsync(w.sys_edge.p, edge.data(), nsys * sizeof(float4), cudaMemcpyHostToDevice,
                     h->st),
     "systems upload");
  CK(cudaMemcpyAsync(b.geoms_dev.p, b.geoms.data(), nsys * sizeof(CellGeom),
                     cudaMemcpyHostToDevice, h->st),
     "systems upload");
  CK(cudaMemcpyAsync(w.xref.p, w.x.p, sizeof(double) * 3 * w.n, cudaMemcpyDeviceToDevice, h->st),
     "xref");
  CK(cudaStreamSynchronize(h->st), "systems upload");
  return DP_OK;
}

// forces, per-atom energies and per-tile virial rows of all the systems
dp_status evaluate_batch(dp_handle* h, Work& w, Batch& b) {
  const int64_t n = w.n;
  if (n == 0) return DP_OK;
  const EnvParams ep = env_params(h);
  launch_zero_forces(h->st, n, P<unsigned long long>(w.ffix));
  CK(cudaMemsetAsync(w.pairs.p, 0, sizeof(unsigned long long), h->st), "memset");
  {
    Phase ph(h, 1);
    if (launch_tab_fwd_tc(h->st, b.tm, P<float4>(w.off), P<uint32_t>(w.nlist), P<int32_t>(w.nn),
                          w.cap, w.geom, ep, P<__nv_bfloat16>(h->tabF), P<float>(h->tc_scratch),
                          P<float4>(w.tc_pairs), P<uint16_t>(w.tc_hist), P<int2>(w.tc_range),
                          P<float>(w.T), P<int32_t>(h->status), P<unsigned long long>(w.pairs),
                          P<int32_t>(w.sys_of), P<int32_t>(w.sys_base), P<float4>(w.sys_edge),
                          fwd_tc_wait_limit()))
      return fail(h, DP_ERR_UNIMPLEMENTED, "tensor-core embedding cannot run this model shape");
  }
  {
    Phase ph(h, 2);
    for (int t = 0; t < h->ntypes; ++t) {
      const int64_t cnt = w.have_idx ? w.type_count[t] : n;
      if (cnt == 0) continue;
      const int32_t* idx = w.have_idx ? P<int32_t>(w.idx) + w.type_off[t] : nullptr;
      CKS(run_fitting(h, t, cnt, idx, P<float>(w.T), P<float>(w.dT), P<double>(w.e_atom)));
      if (!w.have_idx) break;
    }
  }
  {
    Phase ph(h, 3);
    if (launch_tab_bwd_tc(h->st, b.tm, P<float4>(w.tc_pairs), P<uint16_t>(w.tc_hist),
                          P<int2>(w.tc_range), ep, P<__nv_bfloat16>(h->tabB), P<float>(w.dT),
                          P<unsigned long long>(w.ffix), P<double>(w.vir_part),
                          (int)tab_tc_slots(), P<int32_t>(h->status), P<double>(w.vir_tile)))
      return fail(h, DP_ERR_UNIMPLEMENTED, "tensor-core embedding cannot run this model shape");
  }
  launch_force_finalize(h->st, n, P<unsigned long long>(w.ffix), P<double>(w.f),
                        P<int32_t>(h->status));
  launch_check_energy(h->st, n, P<double>(w.e_atom), P<int32_t>(h->status));
  CK(cudaGetLastError(), "evaluation kernels");
  return DP_OK;
}

// Per-system sums of a batch, each bitwise the one the system has alone: its
// atoms' energies (segments of e_atom; of the kinetic terms likewise) and,
// per centre type, its tiles' virial rows (segments of vir_tile), added in
// type order.  The segment table (rows of each segment, then its first row:
// systems, then (system, type) tile ranges) goes to w.seg; *nvseg is the
// number of tile ranges.
static dp_status batch_seg_upload(dp_handle* h, Work& w, const Batch& b, int* nvseg) {
  const int nsys = b.nsys;
  std::vector<int64_t> seg;
  int nv = 0;
  for (int q = 0; q < nsys; ++q) seg.push_back(b.base[q + 1] - b.base[q]);
  for (int q = 0; q < nsys; ++q)
    for (auto& r : b.sys_tiles[q]) seg.push_back(r.second), ++nv;
  for (int q = 0; q < nsys; ++q) seg.push_back(b.base[q]);
  for (int q = 0; q < nsys; ++q)
    for (auto& r : b.sys_tiles[q]) seg.push_back(r.first);
  *nvseg = nv;
  CK(ensure(w.seg, std::max<size_t>(seg.size(), 1) * sizeof(int64_t)), "alloc sums");
  CK(ensure(w.seg_part, (size_t)std::max<int64_t>(sum_rows_seg_part_size(nsys, 1),
                                                   sum_rows_seg_part_size(nv, 9)) *
                            sizeof(double)),
     "alloc sums");
  if (!seg.empty())
    CK(cudaMemcpyAsync(w.seg.p, seg.data(), seg.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                       h->st),
       "sums upload");
  return DP_OK;
}

// doubles of one record of batch_seg_launch: [nsys] energies, [nvseg][9]
// virial rows, then (with kinetic terms) [nsys] kinetic sums
static size_t batch_seg_len(const Batch& b, int nvseg, bool ke) {
  return (size_t)b.nsys * (ke ? 2 : 1) + 9 * (size_t)nvseg;
}

// the sums of batch_seg_upload's table into out (device, batch_seg_len)
static void batch_seg_launch(dp_handle* h, Work& w, const Batch& b, int nvseg,
                             const double* ke, double* out) {
  const int nsys = b.nsys;
  const int64_t* rows = P<int64_t>(w.seg);
  const int64_t* offs = rows + nsys + nvseg;
  launch_sum_rows_seg(h->st, nsys, rows, offs, 1, P<double>(w.e_atom), P<double>(w.seg_part),
                      out);
  launch_sum_rows_seg(h->st, nvseg, rows + nsys, offs + nsys, 9, P<double>(w.vir_tile),
                      P<double>(w.seg_part), out + nsys);
  if (ke)
    launch_sum_rows_seg(h->st, nsys, rows, offs, 1, ke, P<double>(w.seg_part),
                        out + nsys + 9 * (size_t)nvseg);
}

// system q's virial from a record of batch_seg_launch: its tile ranges'
// rows added in order from zero (the order of launch_add_rows)
static void batch_seg_virial(const Batch& b, const double* rec, int q, double* v) {
  size_t vk = 0;
  for (int p = 0; p < q; ++p) vk += b.sys_tiles[p].size();
  for (int a = 0; a < 9; ++a) v[a] = 0.0;
  for (size_t r = 0; r < b.sys_tiles[q].size(); ++r, ++vk)
    for (int a = 0; a < 9; ++a) v[a] += rec[b.nsys + 9 * vk + a];
}

dp_status batch_sums(dp_handle* h, Work& w, Batch& b, double* energies, double* virials) {
  const int nsys = b.nsys;
  int nvseg = 0;
  std::vector<double> out(batch_seg_len(b, 0, false), 0.0);
  if (w.n > 0) {
    CKS(batch_seg_upload(h, w, b, &nvseg));
    out.assign(batch_seg_len(b, nvseg, false), 0.0);
    CK(ensure(w.seg_out, out.size() * sizeof(double)), "alloc sums");
    batch_seg_launch(h, w, b, nvseg, nullptr, P<double>(w.seg_out));
    CK(cudaGetLastError(), "sum kernels");
    CK(cudaMemcpyAsync(out.data(), w.seg_out.p, out.size() * sizeof(double),
                       cudaMemcpyDeviceToHost, h->st),
       "energy copy");
    CK(cudaStreamSynchronize(h->st), "energy copy");
  }
  for (int q = 0; q < nsys; ++q) {
    energies[q] = out[q];
    if (w.n > 0) batch_seg_virial(b, out.data(), q, virials + 9 * q);
    else for (int a = 0; a < 9; ++a) virials[9 * q + a] = 0.0;
  }
  return DP_OK;
}

dp_status check_handle(dp_handle* h) {
  if (!h) return DP_ERR_ARG;
  if (h->dead) return fail(h, DP_ERR_CUDA, "handle unusable after an earlier CUDA error");
  h->err.clear();
  return DP_OK;
}

// The FP16-pair scales of a type's fitting net from its FP32 weights (host
// copy `fb`, the fit32 layout): each a power of two that maps an upper bound
// of the operand's magnitude to at most 2^14 (the FP16 maximum is 65504).
// Weights: their largest |w|.  Forward activations: z_0 = tanh is within 1,
// and a shortcut adds at most 1 per layer.  Gradients: dE/dz of the last
// layer is w_out; through layer k, |dE/dz_{k-1}| <= max_j sum_n |W_k[j][n]|
// max|dE/da_k| (+ max|dE/dz_k| with a shortcut), and |dE/da| <= |dE/dz| d_max
// with d_max >= every |tanh'| (the tanh table's polynomial derivative
// included).
static void fit_pair_scales(const dp_handle* h, int t, const float* fb, FitNetTC& nt) {
  const FitNet& nf = h->nets[t];
  const auto& o = h->fit_ofs[t];
  auto scale_for = [](double bound) {
    if (!(bound > 0.0) || !std::isfinite(bound)) return 1.0f;
    const int e = (int)std::ceil(std::log2(bound));
    return (float)std::ldexp(1.0, std::max(-100, std::min(100, 14 - e)));
  };
  const double dmax = 1.0625;
  double bz = 0.0;
  for (int k = 0; k < nf.nl; ++k) {
    const int wi = nf.win[k], wo = nf.wout[k];
    double wmax = 0.0;
    for (int64_t q = 0; q < (int64_t)wi * wo; ++q)
      wmax = std::max(wmax, (double)std::fabs(fb[o.W[k] + q]));
    nt.s_w[k] = nt.s_wt[k] = scale_for(wmax);
    bz = (k > 0 && nf.shortcut[k] ? bz : 0.0) + 1.0;
    nt.s_z[k] = scale_for(bz);
  }
  const int nl = nf.nl, wl = nf.wout[nl - 1];
  double bgz = 0.0;
  for (int c = 0; c < wl; ++c) bgz = std::max(bgz, (double)std::fabs(fb[o.wout + c]));
  double bgp = bgz * dmax;
  nt.s_g[nl - 1] = scale_for(bgp);
  for (int k = nl - 1; k >= 1; --k) {
    const int wi = nf.win[k], wo = nf.wout[k];
    double rs = 0.0;
    for (int j = 0; j < wi; ++j) {
      double a = 0.0;
      for (int n = 0; n < wo; ++n) a += std::fabs(fb[o.W[k] + (size_t)j * wo + n]);
      rs = std::max(rs, a);
    }
    bgz = rs * bgp + (nf.shortcut[k] ? bgz : 0.0);
    bgp = bgz * dmax;
    nt.s_g[k - 1] = scale_for(bgp);
  }
}

// pieces of every fitting weight (W^T and W, pre-tiled B operands of the
// tensor-core fitting) from the FP32 copies in fit32 (fb: their host copy,
// for the FP16-pair scales)
// The plain path's FP32 embedding weights, from the embedding nets' FP64
// parameters in the model file's layout (per (centre, neighbor) type pair,
// per layer W then b, contiguous): every sub-array padded to a 16-byte
// boundary (the kernels read float4), plus the transposes the backward
// reads, and one device record per pair pointing into them.
static dp_status upload_plain_nets(dp_handle* h, const double* emb) {
  const int d1 = h->emb_w[0], d2 = h->emb_w[1], Me = h->emb_w[2];
  const int np = h->ntypes * h->ntypes;
  auto pad4 = [](size_t v) { return (v + 3) & ~(size_t)3; };
  const size_t oW0 = 0, ob0 = pad4(d1), oW1 = ob0 + pad4(d1), ob1 = oW1 + pad4((size_t)d1 * d2),
               oW2 = ob1 + pad4(d2), ob2 = oW2 + pad4((size_t)d2 * Me),
               oW1T = ob2 + pad4(Me), oW2T = oW1T + pad4((size_t)d1 * d2),
               per = oW2T + pad4((size_t)d2 * Me);
  const size_t pair_doubles = (size_t)plain_wgrad_params(d1, Me);
  std::vector<float> pw((size_t)np * per, 0.0f);
  for (int p = 0; p < np; ++p) {
    float* q = pw.data() + (size_t)p * per;
    const double* W0 = emb + (size_t)p * pair_doubles;  // W0[d1], b0[d1]
    const double* W1 = W0 + 2 * d1;                     // W1[d1][d2], b1[d2]
    const double* W2 = W1 + (size_t)(d1 + 1) * d2;      // W2[d2][Me], b2[Me]
    for (int k = 0; k < d1; ++k) {
      q[oW0 + k] = (float)W0[k];
      q[ob0 + k] = (float)W0[d1 + k];
    }
    for (size_t k = 0; k < (size_t)d1 * d2; ++k) q[oW1 + k] = (float)W1[k];
    for (int k = 0; k < d2; ++k) q[ob1 + k] = (float)W1[(size_t)d1 * d2 + k];
    for (size_t k = 0; k < (size_t)d2 * Me; ++k) q[oW2 + k] = (float)W2[k];
    for (int k = 0; k < Me; ++k) q[ob2 + k] = (float)W2[(size_t)d2 * Me + k];
    for (int mm = 0; mm < d2; ++mm)
      for (int k = 0; k < d1; ++k) q[oW1T + (size_t)mm * d1 + k] = (float)W1[(size_t)k * d2 + mm];
    for (int c = 0; c < Me; ++c)
      for (int l = 0; l < d2; ++l) q[oW2T + (size_t)c * d2 + l] = (float)W2[(size_t)l * Me + c];
  }
  const size_t rb = plain_net_bytes();
  std::vector<unsigned char> recs((size_t)np * rb);
  if (ensure(h->plain_w, sizeof(float) * pw.size()) != cudaSuccess ||
      cudaMemcpyAsync(h->plain_w.p, pw.data(), sizeof(float) * pw.size(), cudaMemcpyHostToDevice,
                      h->st) != cudaSuccess) {
    h->err = "device allocation failed";
    cudaGetLastError();
    return DP_ERR_OOM;
  }
  const float* dpw = P<float>(h->plain_w);
  for (int p = 0; p < np; ++p) {
    const float* b = dpw + (size_t)p * per;
    if (!plain_net_fill(recs.data() + (size_t)p * rb, b + oW0, b + ob0, b + oW1, b + ob1,
                        b + oW2, b + ob2, b + oW1T, b + oW2T) ||
        Me % 4) {
      h->err = "plain embedding weights are not 16-byte aligned";
      return DP_ERR_UNIMPLEMENTED;
    }
  }
  if (ensure(h->plain_nets, recs.size()) != cudaSuccess ||
      cudaMemcpyAsync(h->plain_nets.p, recs.data(), recs.size(), cudaMemcpyHostToDevice,
                      h->st) != cudaSuccess ||
      cudaStreamSynchronize(h->st) != cudaSuccess) {
    h->err = "device allocation failed";
    cudaGetLastError();
    return DP_ERR_OOM;
  }
  return DP_OK;
}

void tile_fit_weights(dp_handle* h, const float* host_fb) {
  const float* fb = P<float>(h->fit32);
  __nv_bfloat16* hb = P<__nv_bfloat16>(h->fit_bf16);
  const int pcode = fit_pieces(h->opt.fit_precision);  // fit_precision 0: unused
  const int pc = pcode == 4 ? 3 : pcode;
  for (int t = 0; t < h->ntypes; ++t) {
    const FitNet& nf = h->nets[t];
    FitNetTC& nt = h->nets_tc[t];
    const auto& o = h->fit_ofs[t];
    for (int k = 0; k < DP_MAXFIT; ++k) nt.s_wt[k] = nt.s_w[k] = nt.s_z[k] = nt.s_g[k] = 1.0f;
    if (pcode == 2 || pcode == 4) fit_pair_scales(h, t, host_fb, nt);
    for (int k = 0; k < nf.nl; ++k)
      if (nf.wout[k] % 16 == 0 && nf.win[k] % 16 == 0) {
        // W^T (N = wout, K = win), W (N = win, K = wout)
        launch_tile_operand(h->st, nf.wout[k], nf.win[k], pc, nt.s_wt[k], fb + o.WT[k],
                            hb + 3 * o.WT[k]);
        // W_0 is the dE/dD GEMM's B operand: an FP16 pair in the mixed mode
        launch_tile_operand(h->st, nf.win[k], nf.wout[k], pcode == 4 && k == 0 ? 2 : pc,
                            nt.s_w[k], fb + o.W[k], hb + 3 * o.W[k]);
      }
  }
}

// copy in x (host or device) and user types; returns model types on device
dp_status load_coords(dp_handle* h, Work& w, int64_t n, const double* coords,
                      const int32_t* types, int device_ptrs) {
  CKS(ensure_atoms(h, w, n));
  if (n == 0) return DP_OK;
  const cudaMemcpyKind kind = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(w.x.p, coords, sizeof(double) * 3 * n, kind, h->st), "coords copy");
  std::vector<int32_t> th;
  const int32_t* types_host = types;
  if (device_ptrs) {
    th.resize(n);
    CK(cudaMemcpyAsync(th.data(), types, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, h->st),
       "types copy");
    CK(cudaStreamSynchronize(h->st), "types copy");
    types_host = th.data();
  }
  return set_types(h, w, types_host);
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

void dp_options_default(dp_options* o) {
  if (!o) return;
  o->tabulated = 1;
  o->fit_precision = 0;
  o->table_step = 0.01;
  o->s_max = 2.0;
  o->skin = 2.0;
  o->rebuild_every = 10;
  o->embed_precision = 0;
  o->tanh_table = 0;
  o->md_graphs = 1;
  o->s_ext = 0.0;
  o->ext_stride = 10;
}

const char* dp_version(void) {
  return "dp-gb300 0.2 (sm_103a; tabulated embedding and fitting net on FP32 CUDA cores or "
         "tcgen05 tensor cores)";
}

const char* dp_last_error(const dp_handle* h) { return h ? h->err.c_str() : g_create_err.c_str(); }

dp_status dp_set_stream(dp_handle* h, void* stream) {
  if (!h) return DP_ERR_ARG;
  h->st = (cudaStream_t)stream;
  return DP_OK;
}

dp_status dp_create(const char* model_path, int ntypes, const int32_t* type_map, double rc,
                    double rcs, const int32_t* sel, const dp_options* opt, void* stream,
                    dp_handle** out) {
  if (!out) return DP_ERR_ARG;
  *out = nullptr;
  dp_handle* h = new dp_handle();
  g_create_err.clear();
  auto bail = [&](dp_status s) {
    g_create_err = h->err.empty() ? "dp_create failed" : h->err;
    if (h->status_host) cudaFreeHost(h->status_host);
    delete h;
    return s;
  };
  h->st = (cudaStream_t)stream;
  if (opt)
    h->opt = *opt;
  else
    dp_options_default(&h->opt);
  if (!model_path || !sel || ntypes < 1 || ntypes > DP_MAXT || !(rc > 0) || !(rcs >= 0) ||
      !(rcs < rc) || !(h->opt.table_step > 0) || !(h->opt.s_max > 0) || h->opt.skin < 0 ||
      h->opt.rebuild_every < 1)
    return bail(DP_ERR_ARG);
  if (h->opt.tabulated < 0 || h->opt.tabulated > 1 || h->opt.fit_precision < 0 ||
      h->opt.fit_precision > 4 || (h->opt.embed_precision != 0 && h->opt.embed_precision != 2) ||
      h->opt.tanh_table < 0 || h->opt.tanh_table > 1 || h->opt.md_graphs < 0 ||
      h->opt.md_graphs > 1)
    return bail(DP_ERR_UNIMPLEMENTED);
  if (h->opt.ext_stride < 1 || h->opt.ext_stride > 1000 || !(h->opt.s_ext >= 0.0))
    return bail(DP_ERR_ARG);
  HostModel m;
  std::string why;
  if (!read_model(model_path, m, why)) {
    h->err = why;
    return bail(DP_ERR_MODEL);
  }
  h->ntypes = m.ntypes;
  h->n_emb = m.n_emb;
  for (int k = 0; k < m.n_emb; ++k) h->emb_w[k] = m.emb_w[k];
  h->M = m.emb_w[m.n_emb - 1];
  h->m_lt = m.m_lt;
  h->din = h->M * h->m_lt;
  h->n_fit = m.n_fit;
  for (int k = 0; k < m.n_fit; ++k) h->fit_w[k] = m.fit_w[k];
  if (h->din % 16) return bail(DP_ERR_UNIMPLEMENTED);
  for (int k = 0; k < m.n_fit; ++k)
    if (h->fit_w[k] % 16) return bail(DP_ERR_UNIMPLEMENTED);
  h->ntypes_user = ntypes;
  for (int t = 0; t < ntypes; ++t) {
    h->type_map[t] = type_map ? type_map[t] : t;
    if (h->type_map[t] < 0 || h->type_map[t] >= m.ntypes) return bail(DP_ERR_ARG);
  }
  h->rc = rc;
  h->rcs = rcs;
  h->Nm = 0;
  for (int t = 0; t < m.ntypes; ++t) {
    if (sel[t] < 0) return bail(DP_ERR_ARG);
    h->sel[t] = sel[t];
    h->Nm += sel[t];
  }
  if (h->Nm <= 0) return bail(DP_ERR_ARG);
  h->h = h->opt.table_step;
  h->n_fine = std::max(1, (int)std::ceil(h->opt.s_max / h->h - 1e-9));
  h->H = h->opt.ext_stride * h->h;
  {
    const double rest = h->opt.s_ext - h->n_fine * h->h;
    const double n_ext = rest > 0.0 ? std::ceil(rest / h->H - 1e-9) : 0.0;
    if (n_ext > 4096) return bail(DP_ERR_ARG);
    h->n_int = h->n_fine + (int)n_ext;
  }
  if (h->n_int > 4096) return bail(DP_ERR_ARG);
  if (cudaMallocHost(&h->status_host, sizeof(int32_t) * ST_NWORDS) != cudaSuccess) {
    cudaGetLastError();
    return bail(DP_ERR_OOM);
  }
  auto up = [&](DevBuf& b, const void* src, size_t bytes) -> bool {
    if (ensure(b, bytes) != cudaSuccess) return false;
    return cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, h->st) == cudaSuccess;
  };
  // embedding parameters (FP64, for the table builder)
  const int np = m.ntypes * m.ntypes;
  const int64_t emb_end = m.fit_off.empty() ? (int64_t)m.data.size() : m.fit_off[0];
  bool ok = up(h->emb64, m.data.data(), sizeof(double) * emb_end) &&
            up(h->emb_off, m.emb_off.data(), sizeof(int64_t) * m.emb_off.size()) &&
            up(h->sel_dev, h->sel, sizeof(int32_t) * DP_MAXT) &&
            ensure(h->status, sizeof(int32_t) * ST_NWORDS) == cudaSuccess &&
            ensure(h->table, sizeof(float) * (size_t)np * h->n_int * 6 * h->M) == cudaSuccess;
  // fitting parameters (FP32, plus transposed weights for the backward)
  std::vector<float> fit;
  h->fit_ofs.assign(m.ntypes, dp_handle::FitOfs{});
  auto& ofs = h->fit_ofs;
  for (int t = 0; t < m.ntypes; ++t) {
    int prev = h->din;
    for (int k = 0; k < m.n_fit; ++k) {
      const int wo = m.fit_w[k];
      const double* W = m.data.data() + m.fit_off[t * (m.n_fit + 1) + k];
      ofs[t].W[k] = fit.size();
      for (int64_t q = 0; q < (int64_t)prev * wo; ++q) fit.push_back((float)W[q]);
      ofs[t].WT[k] = fit.size();
      for (int c = 0; c < wo; ++c)
        for (int r = 0; r < prev; ++r) fit.push_back((float)W[(size_t)r * wo + c]);
      ofs[t].b[k] = fit.size();
      for (int c = 0; c < wo; ++c) fit.push_back((float)W[(size_t)prev * wo + c]);
      prev = wo;
    }
    const double* wo_p = m.data.data() + m.fit_off[t * (m.n_fit + 1) + m.n_fit];
    ofs[t].wout = fit.size();
    for (int c = 0; c < prev; ++c) fit.push_back((float)wo_p[c]);
    h->b_out[t] = (float)wo_p[prev];
    while (fit.size() % 4) fit.push_back(0.0f);
  }
  ok = ok && up(h->fit32, fit.data(), sizeof(float) * fit.size());
  h->fit_floats = fit.size();
  if (h->opt.tanh_table) {
    // Sec. 3.5: on [x_k, x_k + h], h = 1/128, p(u) = a0 + a1 u + a2 u^2 with
    // p(0) = tanh(x_k), p'(0) = 1 - tanh(x_k)^2, p(h) = tanh(x_k + h); FP64
    // coefficients rounded to FP32
    std::vector<float> tt(4 * 1024);
    const double hh = 1.0 / 128.0;
    for (int k = 0; k < 1024; ++k) {
      const double y0 = std::tanh(k * hh), y1 = std::tanh((k + 1) * hh);
      const double a1 = 1.0 - y0 * y0;
      tt[4 * k] = (float)y0;
      tt[4 * k + 1] = (float)a1;
      tt[4 * k + 2] = (float)((y1 - y0 - a1 * hh) / (hh * hh));
      tt[4 * k + 3] = 0.0f;
    }
    ok = ok && up(h->tanh_tab, tt.data(), sizeof(float) * tt.size());
  }
  if (!ok) {
    h->err = "device allocation or upload failed";
    cudaGetLastError();
    return bail(DP_ERR_OOM);
  }
  float* fb = P<float>(h->fit32);
  for (int t = 0; t < m.ntypes; ++t) {
    FitNet& net = h->nets[t];
    net.nl = m.n_fit;
    int prev = h->din;
    for (int k = 0; k < m.n_fit; ++k) {
      net.win[k] = prev;
      net.wout[k] = m.fit_w[k];
      net.shortcut[k] = (k > 0 && m.fit_w[k] == prev) ? 1 : 0;
      net.W[k] = fb + ofs[t].W[k];
      net.WT[k] = fb + ofs[t].WT[k];
      net.b[k] = fb + ofs[t].b[k];
      prev = m.fit_w[k];
    }
    net.w_out = fb + ofs[t].wout;
    net.b_out = h->b_out[t];
    net.tanh_tab = h->opt.tanh_table ? P<float4>(h->tanh_tab) : nullptr;
  }
  // BF16 pieces (h, m, l) of the fitting weights for the tensor-core modes
  if (ensure(h->fit_bf16, sizeof(__nv_bfloat16) * 3 * fit.size()) != cudaSuccess) {
    h->err = "device allocation failed";
    cudaGetLastError();
    return bail(DP_ERR_OOM);
  }
  {
    __nv_bfloat16* hb = P<__nv_bfloat16>(h->fit_bf16);
    for (int t = 0; t < m.ntypes; ++t) {
      FitNetTC& nt = h->nets_tc[t];
      const FitNet& nf = h->nets[t];
      nt.nl = nf.nl;
      for (int k = 0; k < nf.nl; ++k) {
        // pieces of W^T at 3*ofs.WT, pieces of W at 3*ofs.W (disjoint: 3 * fit.size() total)
        __nv_bfloat16* pwt = hb + 3 * ofs[t].WT[k];
        __nv_bfloat16* pw = hb + 3 * ofs[t].W[k];
        nt.win[k] = nf.win[k];
        nt.wout[k] = nf.wout[k];
        nt.shortcut[k] = nf.shortcut[k];
        nt.WTh[k] = pwt;
        nt.Wh[k] = pw;
        nt.b[k] = nf.b[k];
      }
      nt.w_out = nf.w_out;
      nt.b_out = nf.b_out;
      nt.tanh_tab = nf.tanh_tab;
    }
    tile_fit_weights(h, fit.data());
  }
  // FP32 embedding weights (and transposes) for the plain untabulated path
  if (m.n_emb == 3 && m.emb_w[0] <= 32) {
    const dp_status st = upload_plain_nets(h, m.data.data());
    if (st != DP_OK) return bail(st);
  } else if (h->opt.tabulated == 0) {
    h->err = "the plain path needs three doubling embedding layers with d1 <= 32";
    return bail(DP_ERR_UNIMPLEMENTED);
  }
  if (table_build(h->st, P<double>(h->emb64), P<int64_t>(h->emb_off), m.n_emb, m.emb_w, np, h->h,
                  h->n_int, h->n_fine, h->H, P<float>(h->table)) != 0) {
    h->err = "table build failed";
    return bail(DP_ERR_CUDA);
  }
  if (h->opt.tabulated && h->opt.embed_precision == 2) {
    const EnvParams ep = env_params(h);
    const int sup = tab_tc_supported(ep);
    if (sup) {
      h->err = sup == -1 ? "tensor-core embedding needs M <= 128, M % 4 == 0"
                         : "tensor-core embedding: ntypes x table intervals too large for the "
                           "shared-memory histograms (lower s_max or raise table_step)";
      return bail(DP_ERR_UNIMPLEMENTED);
    }
    const size_t nt = (size_t)tab_tc_elems(ep) * sizeof(__nv_bfloat16);
    if (ensure(h->tabF, nt) != cudaSuccess || ensure(h->tabB, nt) != cudaSuccess ||
        ensure(h->tc_scratch, (size_t)tab_tc_scratch_floats(ep) * sizeof(float)) != cudaSuccess) {
      h->err = "device allocation failed";
      cudaGetLastError();
      return bail(DP_ERR_OOM);
    }
    if (tab_tc_build(h->st, P<float>(h->table), ep, P<__nv_bfloat16>(h->tabF),
                     P<__nv_bfloat16>(h->tabB)) != 0) {
      h->err = "the tensor-core embedding cannot run this model shape (M <= 128, M % 4 == 0)";
      return bail(DP_ERR_UNIMPLEMENTED);
    }
  }
  if (cudaStreamSynchronize(h->st) != cudaSuccess) {
    h->err = "device error during dp_create";
    return bail(DP_ERR_CUDA);
  }
  *out = h;
  return DP_OK;
}

void dp_destroy(dp_handle* h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  if (h->status_host) cudaFreeHost(h->status_host);
  delete h;
}

dp_status dp_compute(dp_handle* h, int64_t natoms, const double* coords, const int32_t* types,
                     const double* box, int device_ptrs, double* energy, double* forces,
                     double* virial, double* atom_energy) {
  CKS(check_handle(h));
  if (natoms < 0 || !box || !energy || !virial || (natoms > 0 && (!coords || !types || !forces)))
    return fail(h, DP_ERR_ARG, "null pointer or negative atom count");
  if (natoms >= (1LL << 27)) return fail(h, DP_ERR_ARG, "at most 2^27 atoms per call");
  double L[3];
  double box_h[9];
  if (device_ptrs) {
    CK(cudaMemcpy(box_h, box, sizeof box_h, cudaMemcpyDeviceToHost), "box copy");
  } else {
    std::memcpy(box_h, box, sizeof box_h);
  }
  CKS(box_lengths(h, box_h, L));
  Work& w = h->w;
  CKS(load_coords(h, w, natoms, coords, types, device_ptrs));
  CKS(clear_status(h));
  CKS(rebuild(h, w, L, h->rc));
  CKS(status_errors(h));
  CKS(evaluate(h, w));
  CKS(read_status(h));
  CKS(status_errors(h));
  const int64_t n = natoms;
  const cudaMemcpyKind kind = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CK(cudaMemcpyAsync(energy, w.red_out.p, sizeof(double), kind, h->st), "energy copy");
  CK(cudaMemcpyAsync(virial, P<double>(w.red_out) + 1, 9 * sizeof(double), kind, h->st),
     "virial copy");
  if (n > 0) {
    CK(cudaMemcpyAsync(forces, w.f.p, sizeof(double) * 3 * n, kind, h->st), "force copy");
    if (atom_energy)
      CK(cudaMemcpyAsync(atom_energy, w.e_atom.p, sizeof(double) * n, kind, h->st), "e copy");
  }
  if (!device_ptrs) CK(cudaStreamSynchronize(h->st), "result copy");
  return DP_OK;
}

dp_status dp_compute_batch(dp_handle* h, int nsys, const int64_t* natoms, const double* coords,
                           const int32_t* types, const double* boxes, double* energies,
                           double* forces, double* virials) {
  CKS(check_handle(h));
  if (nsys > 0 && (!energies || !virials)) return fail(h, DP_ERR_ARG, "bad argument");
  Batch b;
  CKS(batch_init(h, b, nsys, natoms, boxes));
  const int64_t n = b.base[nsys];
  if (n > 0 && (!coords || !types || !forces)) return fail(h, DP_ERR_ARG, "null pointer");
  Work& w = h->w;
  CKS(load_coords(h, w, n, coords, types, 0));
  CKS(clear_status(h));
  CKS(batch_tiles(h, w, b, types));
  CKS(batch_rebuild(h, w, b, h->rc));
  CKS(status_errors(h));
  CKS(evaluate_batch(h, w, b));
  CKS(read_status(h));
  CKS(status_errors(h));
  CKS(batch_sums(h, w, b, energies, virials));
  if (n > 0) {
    CK(cudaMemcpyAsync(forces, w.f.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, h->st),
       "force copy");
    CK(cudaStreamSynchronize(h->st), "force copy");
  }
  return DP_OK;
}

dp_status dp_neighbor_pairs(dp_handle* h, int64_t natoms, const double* coords, const double* box,
                            double rlist, int64_t cap, int32_t* out5, int64_t* count) {
  CKS(check_handle(h));
  if (natoms < 0 || !box || !count || (natoms > 0 && !coords) || !(rlist > 0))
    return fail(h, DP_ERR_ARG, "bad argument");
  double L[3];
  CKS(box_lengths(h, box, L));
  Work& w = h->w;
  std::vector<int32_t> zeros(natoms, 0);
  // all atoms as caller type 0 (the list does not depend on types)
  CKS(ensure_atoms(h, w, natoms));
  if (natoms)
    CK(cudaMemcpyAsync(w.x.p, coords, sizeof(double) * 3 * natoms, cudaMemcpyHostToDevice, h->st),
       "coords copy");
  CKS(set_types(h, w, zeros.data()));
  CKS(clear_status(h));
  CKS(rebuild(h, w, L, rlist));
  const int64_t n = natoms;
  std::vector<uint32_t> nl((size_t)n * w.cap);
  std::vector<int32_t> nn(n), cellc(n);
  if (n) {
    CK(cudaMemcpy(nl.data(), w.nlist.p, sizeof(uint32_t) * nl.size(), cudaMemcpyDeviceToHost),
       "list copy");
    CK(cudaMemcpy(nn.data(), w.nn.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost), "list copy");
    CK(cudaMemcpy(cellc.data(), w.cellc.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost),
       "list copy");
  }
  const CellGeom& g = w.geom;
  int64_t k = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int id = cellc[i];
    const int ci[3] = {id / (g.nc[2] * g.nc[1]), (id / g.nc[2]) % g.nc[1], id % g.nc[2]};
    for (int q = 0; q < std::min(nn[i], w.cap); ++q, ++k) {
      if (k >= cap || !out5) continue;
      const uint32_t e = nl[(size_t)i * w.cap + q];
      const int slot = e & 31;
      const int o[3] = {slot / 9 - 1, (slot / 3) % 3 - 1, slot % 3 - 1};
      int32_t* r = out5 + k * 5;
      r[0] = (int32_t)i;
      r[1] = (int32_t)(e >> 5);
      for (int a = 0; a < 3; ++a) {
        const int v = ci[a] + o[a];
        r[2 + a] = v < 0 ? -1 : (v >= g.nc[a] ? 1 : 0);
      }
    }
  }
  *count = k;
  return DP_OK;
}

dp_status dp_table_coeffs(dp_handle* h, int ti, int tj, float* out, int32_t* n) {
  CKS(check_handle(h));
  if (ti < 0 || tj < 0 || ti >= h->ntypes || tj >= h->ntypes) return fail(h, DP_ERR_ARG, "type");
  if (n) *n = h->n_int;
  if (!out) return DP_OK;
  const size_t sz = (size_t)h->n_int * 6 * h->M;
  CK(cudaMemcpy(out, P<float>(h->table) + (size_t)(ti * h->ntypes + tj) * sz, sz * sizeof(float),
                cudaMemcpyDeviceToHost),
     "table copy");
  return DP_OK;
}

dp_status dp_descriptor(dp_handle* h, int64_t natoms, const double* coords, const int32_t* types,
                        const double* box, float* T_out) {
  CKS(check_handle(h));
  if (natoms < 0 || !box || (natoms > 0 && (!coords || !types || !T_out)))
    return fail(h, DP_ERR_ARG, "bad argument");
  double L[3];
  CKS(box_lengths(h, box, L));
  Work& w = h->w;
  CKS(load_coords(h, w, natoms, coords, types, 0));
  CKS(clear_status(h));
  CKS(rebuild(h, w, L, h->rc));
  CKS(status_errors(h));
  if (natoms == 0) return DP_OK;
  const EnvParams ep = env_params(h);
  CKS(embed_forward(h, w, ep));
  CKS(read_status(h));
  CKS(status_errors(h));
  CK(cudaMemcpy(T_out, w.T.p, sizeof(float) * 4 * h->M * natoms, cudaMemcpyDeviceToHost),
     "T copy");
  return DP_OK;
}

dp_status dp_profile(dp_handle* h, int enable) {
  if (!h) return DP_ERR_ARG;
  for (auto& v : h->prof_ev) {
    for (auto& e : v) h->prof_pool.push_back(e);
    v.clear();
  }
  h->prof = enable != 0;
  return DP_OK;
}

dp_status dp_profile_read(dp_handle* h, double* ms, int64_t* launches) {
  CKS(check_handle(h));
  CK(cudaStreamSynchronize(h->st), "sync");
  for (int p = 0; p < DP_NPHASE; ++p) {
    double t = 0.0;
    for (auto& e : h->prof_ev[p]) {
      float x = 0.0f;
      CK(cudaEventElapsedTime(&x, e.first, e.second), "event time");
      t += x;
    }
    if (ms) ms[p] = t;
    if (launches) launches[p] = (int64_t)h->prof_ev[p].size();
  }
  return DP_OK;
}

dp_status dp_memory(const dp_handle* h, int64_t* handle_bytes, int64_t* process_bytes,
                    int64_t* process_peak, int reset_peak) {
  if (handle_bytes) {
    if (!h) return DP_ERR_ARG;
    const DevBuf* own[] = {&h->emb64,  &h->emb_off,  &h->table,      &h->fit32,    &h->sel_dev,
                           &h->map_dev, &h->status,  &h->tabF,       &h->tabB,     &h->tc_scratch,
                           &h->tanh_tab, &h->pg,     &h->pg_fit_part, &h->pg_tab_part,
                           &h->fitbuf,  &h->fit_bf16, &h->fitbuf_tc, &h->plain_w,  &h->plain_nets,
                           &h->spare_v};
    size_t b = h->w.bytes() + (h->spare_work ? h->spare_work->bytes() : 0);
    for (const DevBuf* d : own) b += d->bytes;
    *handle_bytes = (int64_t)b;
  }
  if (process_bytes) *process_bytes = g_dev_bytes.load();
  if (process_peak) *process_peak = g_dev_peak.load();
  if (reset_peak) g_dev_peak.store(g_dev_bytes.load());
  return DP_OK;
}

dp_status dp_trim(dp_handle* h) {
  CKS(check_handle(h));
  CK(cudaStreamSynchronize(h->st), "sync");
  // the work area of dp_compute, the buffers kept from destroyed systems and
  // the fitting and gradient scratch; all are allocated again on demand
  h->w = Work();
  h->spare_work.reset();
  h->spare_v.release();
  h->fitbuf.release();
  h->fs = FitScratch{};
  h->fitbuf_tc.release();
  h->fs_tc = FitScratchTC{};
  h->pg.release();
  h->pg_fit_part.release();
  h->pg_tab_part.release();
  // CUDA graphs captured by live systems may point into the scratch
  g_alloc_gen.fetch_add(1);
  return DP_OK;
}

dp_status dp_stats(dp_handle* h, const dp_system* s, int64_t* out) {
  CKS(check_handle(h));
  if (!out) return fail(h, DP_ERR_ARG, "null output");
  Work& w = s ? const_cast<dp_system*>(s)->w : h->w;
  unsigned long long pairs = 0;
  if (w.pairs.p) {
    CK(cudaStreamSynchronize(h->st), "sync");
    CK(cudaMemcpy(&pairs, w.pairs.p, sizeof pairs, cudaMemcpyDeviceToHost), "stats copy");
  }
  CKS(read_status(h));
  out[0] = w.n;
  out[1] = w.cap;
  out[2] = h->status_host[ST_MAXLIST];
  out[3] = (int64_t)pairs;
  out[4] = w.geom.ncell;
  out[5] = (int64_t)__atomic_load_n(&g_dp_launches, __ATOMIC_RELAXED);
  return DP_OK;
}

dp_status dp_fitting(dp_handle* h, int64_t natoms, const int32_t* types, const float* T,
                     double* e_out, float* dT_out) {
  CKS(check_handle(h));
  if (natoms < 0 || (natoms > 0 && (!types || !T || !e_out)))
    return fail(h, DP_ERR_ARG, "bad argument");
  if (natoms == 0) return DP_OK;
  Work& w = h->w;
  CKS(ensure_atoms(h, w, natoms));
  CKS(set_types(h, w, types));
  CK(cudaMemcpyAsync(w.T.p, T, sizeof(float) * 4 * h->M * natoms, cudaMemcpyHostToDevice, h->st),
     "T copy");
  CKS(clear_status(h));
  for (int t = 0; t < h->ntypes; ++t) {
    const int64_t cnt = w.have_idx ? w.type_count[t] : natoms;
    if (cnt == 0) continue;
    const int32_t* idx = w.have_idx ? P<int32_t>(w.idx) + w.type_off[t] : nullptr;
    CKS(run_fitting(h, t, cnt, idx, P<float>(w.T), P<float>(w.dT), P<double>(w.e_atom)));
    if (!w.have_idx) break;
  }
  CK(cudaGetLastError(), "fitting kernels");
  CKS(read_status(h));
  CKS(status_errors(h));
  CK(cudaMemcpy(e_out, w.e_atom.p, sizeof(double) * natoms, cudaMemcpyDeviceToHost), "e copy");
  if (dT_out)
    CK(cudaMemcpy(dT_out, w.dT.p, sizeof(float) * 4 * h->M * natoms, cudaMemcpyDeviceToHost),
       "dT copy");
  return DP_OK;
}

// ---------------------------------------------------------------------- MD
static int64_t fit_params_per_type(const dp_handle* h) {
  int64_t c = 0;
  int win = h->din;
  for (int k = 0; k < h->n_fit; ++k) {
    c += (int64_t)(win + 1) * h->fit_w[k];
    win = h->fit_w[k];
  }
  return c + win + 1;
}

// doubles of the embedding representation's gradient: the table
// coefficients (tabulated) or the embedding nets' weights and biases
static int64_t emb_repr_params(const dp_handle* h) {
  const int64_t np = (int64_t)h->ntypes * h->ntypes;
  if (h->opt.tabulated) return np * h->n_int * 6 * h->M;
  return np * plain_wgrad_params(h->emb_w[0], h->M);
}

dp_status dp_param_sizes(dp_handle* h, int64_t* n_fit, int64_t* n_table) {
  CKS(check_handle(h));
  if (n_fit) *n_fit = fit_params_per_type(h) * h->ntypes;
  if (n_table) *n_table = emb_repr_params(h);
  return DP_OK;
}

dp_status dp_param_grad(dp_handle* h, int64_t natoms, const double* coords, const int32_t* types,
                        const double* box, double* energy, double* grad_fit,
                        double* grad_table) {
  CKS(check_handle(h));
  if (natoms < 0 || !box || !energy || !grad_fit || (natoms > 0 && (!coords || !types)))
    return fail(h, DP_ERR_ARG, "null pointer or negative atom count");
  if (natoms >= (1LL << 27)) return fail(h, DP_ERR_ARG, "at most 2^27 atoms per call");
  if (grad_table && h->opt.tabulated && h->opt.embed_precision != 2)
    return fail(h, DP_ERR_UNIMPLEMENTED,
                "table gradients need the tabulated tensor-core embedding (embed_precision 2)");
  double L[3];
  CKS(box_lengths(h, box, L));
  Work& w = h->w;
  CKS(load_coords(h, w, natoms, coords, types, 0));
  CKS(clear_status(h));
  CKS(rebuild(h, w, L, h->rc));
  CKS(status_errors(h));
  const int64_t per = fit_params_per_type(h);
  const int64_t nfit = per * h->ntypes;
  const int64_t ntab = emb_repr_params(h);
  CK(ensure(h->pg, sizeof(double) * (size_t)(nfit + ntab)), "alloc gradients");
  CK(cudaMemsetAsync(h->pg.p, 0, sizeof(double) * (size_t)(nfit + ntab), h->st), "memset");
  const int64_t n = natoms;
  if (n > 0) {
    const EnvParams ep = env_params(h);
    CK(cudaMemsetAsync(w.pairs.p, 0, sizeof(unsigned long long), h->st), "memset");
    CKS(embed_forward(h, w, ep));
    // a forward that gave up leaves no sorted pairs for the table gradient
    CKS(read_status(h));
    CKS(status_errors(h));
    // the fitting stage on the FP32 CUDA-core path, which keeps every
    // layer's input and gradient for the parameter gradients
    for (int t = 0; t < h->ntypes; ++t) {
      const int64_t cnt = w.have_idx ? w.type_count[t] : n;
      if (cnt == 0) continue;
      const int32_t* idx = w.have_idx ? P<int32_t>(w.idx) + w.type_off[t] : nullptr;
      CKS(ensure_fit_scratch(h, cnt));
      const int64_t pf = fit_grad_part_floats(h->nets[t], h->din, h->fs.rows);
      CK(ensure(h->pg_fit_part, sizeof(float) * (size_t)pf), "alloc gradient partials");
      FitGrad fg{P<double>(h->pg) + (size_t)t * per, P<float>(h->pg_fit_part), pf};
      if (fit_simt(h->st, cnt, idx, h->nets[t], h->M, h->m_lt, P<float>(w.T), P<float>(w.dT),
                   P<double>(w.e_atom), h->fs, &fg))
        return fail(h, DP_ERR_CUDA, "fitting kernels failed to launch");
      if (!w.have_idx) break;
    }
    if (grad_table && h->opt.tabulated) {
      const int64_t tp = tab_grad_part_floats(ep);
      CK(ensure(h->pg_tab_part, sizeof(float) * (size_t)tp), "alloc gradient partials");
      if (launch_tab_grad_tc(h->st, w.tiles, P<float4>(w.tc_pairs), P<uint16_t>(w.tc_hist),
                             P<int2>(w.tc_range), ep, P<float>(w.dT), P<float>(h->pg_tab_part),
                             P<double>(h->pg) + nfit))
        return fail(h, DP_ERR_UNIMPLEMENTED, "table gradient cannot run this model shape");
    } else if (grad_table) {
      // the original embedding nets: one launch per (centre, neighbor) type pair
      const int npar = plain_wgrad_params(h->emb_w[0], h->M);
      CK(ensure(h->pg_tab_part, sizeof(float) * (size_t)plain_wgrad_ctas() * npar),
         "alloc gradient partials");
      for (int ti = 0; ti < h->ntypes; ++ti)
        for (int tj = 0; tj < h->ntypes; ++tj)
          if (launch_plain_wgrad(h->st, n, P<float4>(w.off), P<uint32_t>(w.nlist),
                                 P<int32_t>(w.nn), w.cap, w.geom, ep, h->plain_nets.p, h->emb_w[0],
                                 P<float>(w.dT), ti, tj, P<float>(h->pg_tab_part),
                                 P<double>(h->pg) + nfit + (size_t)(ti * h->ntypes + tj) * npar))
            return fail(h, DP_ERR_UNIMPLEMENTED, "embedding-net gradient cannot run this model");
    }
    launch_sum_rows(h->st, n, 1, P<double>(w.e_atom), P<double>(w.red_part), P<double>(w.red_out));
    launch_check_energy(h->st, n, P<double>(w.e_atom), P<int32_t>(h->status));
    CK(cudaGetLastError(), "gradient kernels");
  } else {
    CK(cudaMemsetAsync(w.red_out.p, 0, sizeof(double), h->st), "memset");
  }
  CKS(read_status(h));
  CKS(status_errors(h));
  CK(cudaMemcpyAsync(energy, w.red_out.p, sizeof(double), cudaMemcpyDeviceToHost, h->st),
     "energy copy");
  CK(cudaMemcpyAsync(grad_fit, h->pg.p, sizeof(double) * (size_t)nfit, cudaMemcpyDeviceToHost,
                     h->st),
     "gradient copy");
  if (grad_table)
    CK(cudaMemcpyAsync(grad_table, P<double>(h->pg) + nfit, sizeof(double) * (size_t)ntab,
                       cudaMemcpyDeviceToHost, h->st),
       "gradient copy");
  CK(cudaStreamSynchronize(h->st), "gradient copy");
  return DP_OK;
}

dp_status dp_get_params(dp_handle* h, double* fit, double* table) {
  CKS(check_handle(h));
  if (fit) {
    std::vector<float> fb(h->fit_floats);
    CK(cudaMemcpyAsync(fb.data(), h->fit32.p, sizeof(float) * fb.size(), cudaMemcpyDeviceToHost,
                       h->st),
       "parameter copy");
    CK(cudaStreamSynchronize(h->st), "parameter copy");
    double* o = fit;
    for (int t = 0; t < h->ntypes; ++t) {
      const FitNet& net = h->nets[t];
      const auto& ofs = h->fit_ofs[t];
      for (int k = 0; k < net.nl; ++k) {
        const size_t nw = (size_t)net.win[k] * net.wout[k];
        for (size_t q = 0; q < nw; ++q) *o++ = fb[ofs.W[k] + q];
        for (int c = 0; c < net.wout[k]; ++c) *o++ = fb[ofs.b[k] + c];
      }
      for (int c = 0; c < net.wout[net.nl - 1]; ++c) *o++ = fb[ofs.wout + c];
      *o++ = h->b_out[t];
    }
  }
  if (table && !h->opt.tabulated) {
    // the embedding nets' FP64 weights and biases, in the file's (and the
    // gradient's) layout
    CK(cudaMemcpy(table, h->emb64.p, sizeof(double) * (size_t)emb_repr_params(h),
                  cudaMemcpyDeviceToHost),
       "embedding copy");
  } else if (table) {
    const size_t n = (size_t)h->ntypes * h->ntypes * h->n_int * 6 * h->M;
    std::vector<float> tb(n);
    CK(cudaMemcpy(tb.data(), h->table.p, sizeof(float) * n, cudaMemcpyDeviceToHost),
       "table copy");
    for (size_t q = 0; q < n; ++q) table[q] = tb[q];
  }
  return DP_OK;
}

dp_status dp_set_params(dp_handle* h, const double* fit, const double* table) {
  CKS(check_handle(h));
  // captured MD graphs hold the output bias by value: capture them again
  g_alloc_gen.fetch_add(1);
  if (fit) {
    std::vector<float> fb(h->fit_floats);
    CK(cudaMemcpyAsync(fb.data(), h->fit32.p, sizeof(float) * fb.size(), cudaMemcpyDeviceToHost,
                       h->st),
       "parameter copy");
    CK(cudaStreamSynchronize(h->st), "parameter copy");
    const double* in = fit;
    for (int t = 0; t < h->ntypes; ++t) {
      FitNet& net = h->nets[t];
      const auto& ofs = h->fit_ofs[t];
      for (int k = 0; k < net.nl; ++k) {
        const int wi = net.win[k], wo = net.wout[k];
        for (int r = 0; r < wi; ++r)
          for (int c = 0; c < wo; ++c) {
            const float v = (float)in[(size_t)r * wo + c];
            fb[ofs.W[k] + (size_t)r * wo + c] = v;
            fb[ofs.WT[k] + (size_t)c * wi + r] = v;
          }
        in += (size_t)wi * wo;
        for (int c = 0; c < wo; ++c) fb[ofs.b[k] + c] = (float)in[c];
        in += wo;
      }
      const int wl = net.wout[net.nl - 1];
      for (int c = 0; c < wl; ++c) fb[ofs.wout + c] = (float)in[c];
      h->b_out[t] = (float)in[wl];
      net.b_out = h->b_out[t];
      h->nets_tc[t].b_out = h->b_out[t];
      in += wl + 1;
    }
    CK(cudaMemcpyAsync(h->fit32.p, fb.data(), sizeof(float) * fb.size(), cudaMemcpyHostToDevice,
                       h->st),
       "parameter upload");
    tile_fit_weights(h, fb.data());
    CK(cudaStreamSynchronize(h->st), "parameter upload");
  }
  if (table && !h->opt.tabulated) {
    // the embedding nets (FP64, the file's layout): the plain path's FP32
    // weights, and the handle's table built from them, follow
    CK(cudaMemcpyAsync(h->emb64.p, table, sizeof(double) * (size_t)emb_repr_params(h),
                       cudaMemcpyHostToDevice, h->st),
       "embedding upload");
    CKS(upload_plain_nets(h, table));
    if (table_build(h->st, P<double>(h->emb64), P<int64_t>(h->emb_off), h->n_emb, h->emb_w,
                    h->ntypes * h->ntypes, h->h, h->n_int, h->n_fine, h->H, P<float>(h->table)) != 0)
      return fail(h, DP_ERR_CUDA, "table build failed");
    CK(cudaStreamSynchronize(h->st), "embedding upload");
  } else if (table) {
    const size_t n = (size_t)h->ntypes * h->ntypes * h->n_int * 6 * h->M;
    std::vector<float> tb(n);
    for (size_t q = 0; q < n; ++q) tb[q] = (float)table[q];
    CK(cudaMemcpyAsync(h->table.p, tb.data(), sizeof(float) * n, cudaMemcpyHostToDevice, h->st),
       "table upload");
    if (h->opt.embed_precision == 2 &&
        tab_tc_build(h->st, P<float>(h->table), env_params(h), P<__nv_bfloat16>(h->tabF),
                     P<__nv_bfloat16>(h->tabB)) != 0)
      return fail(h, DP_ERR_CUDA, "table tiling failed");
    CK(cudaStreamSynchronize(h->st), "table upload");
  }
  return DP_OK;
}

dp_status dp_system_create(dp_handle* h, int64_t natoms, const double* x, const double* v,
                           const int32_t* types, const double* mass_of_type, const double* box,
                           int device_ptrs, dp_system** out) {
  CKS(check_handle(h));
  if (!out || natoms < 0 || !box || !mass_of_type || (natoms > 0 && (!x || !v || !types)))
    return fail(h, DP_ERR_ARG, "bad argument");
  *out = nullptr;
  dp_system* s = new dp_system();
  s->h = h;
  auto bail = [&](dp_status st) {
    delete s;
    return st;
  };
  double box_h[9];
  std::vector<double> mass_h(h->ntypes_user);
  if (device_ptrs) {
    if (cudaMemcpy(box_h, box, sizeof box_h, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(mass_h.data(), mass_of_type, sizeof(double) * h->ntypes_user,
                   cudaMemcpyDeviceToHost) != cudaSuccess)
      return bail(fail(h, DP_ERR_ARG, "box/mass copy failed"));
  } else {
    std::memcpy(box_h, box, sizeof box_h);
    std::memcpy(mass_h.data(), mass_of_type, sizeof(double) * h->ntypes_user);
  }
  double L[3];
  dp_status st = box_lengths(h, box_h, L);
  if (st) return bail(st);
  for (double mm : mass_h)
    if (!(mm > 0)) return bail(fail(h, DP_ERR_ARG, "masses must be > 0"));
  std::memcpy(s->box, box_h, sizeof box_h);
  s->mass_user = mass_h;
  if (h->spare_work) {
    s->w = std::move(*h->spare_work);
    h->spare_work.reset();
    s->v = std::move(h->spare_v);
  }
  st = load_coords(h, s->w, natoms, x, types, device_ptrs);
  if (st) return bail(st);
  s->types_user.resize(natoms);
  if (natoms) {
    if (cudaMemcpy(s->types_user.data(), types, sizeof(int32_t) * natoms,
                   device_ptrs ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost) != cudaSuccess)
      return bail(fail(h, DP_ERR_ARG, "types copy failed"));
  }
  // masses per model-mapped atom type are kept per caller type: store a
  // per-atom-type table indexed by the model type only when unambiguous,
  // else per caller type through the mapped types buffer
  std::vector<double> mass_model(DP_MAXT, 0.0), inv_acc(DP_MAXT, 0.0);
  for (int t = 0; t < h->ntypes_user; ++t) {
    const int mt = h->type_map[t];
    if (mass_model[mt] != 0.0 && mass_model[mt] != mass_h[t])
      return bail(fail(h, DP_ERR_UNIMPLEMENTED, "caller types sharing a model type need equal masses"));
    mass_model[mt] = mass_h[t];
  }
  for (int t = 0; t < DP_MAXT; ++t) inv_acc[t] = mass_model[t] > 0 ? kAcc / mass_model[t] : 0.0;
  if (ensure(s->v, sizeof(double) * 3 * std::max<int64_t>(natoms, 1)) != cudaSuccess ||
      ensure(s->mass, sizeof(double) * DP_MAXT) != cudaSuccess ||
      ensure(s->inv_mass_acc, sizeof(double) * DP_MAXT) != cudaSuccess)
    return bail(fail(h, DP_ERR_OOM, "device allocation failed"));
  cudaMemcpyKind kind = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if ((natoms && cudaMemcpyAsync(s->v.p, v, sizeof(double) * 3 * natoms, kind, h->st)) ||
      cudaMemcpyAsync(s->mass.p, mass_model.data(), sizeof(double) * DP_MAXT,
                      cudaMemcpyHostToDevice, h->st) ||
      cudaMemcpyAsync(s->inv_mass_acc.p, inv_acc.data(), sizeof(double) * DP_MAXT,
                      cudaMemcpyHostToDevice, h->st))
    return bail(fail(h, DP_ERR_CUDA, "upload failed"));
  if ((st = clear_status(h))) return bail(st);
  if ((st = rebuild(h, s->w, L, h->rc + h->opt.skin))) return bail(st);
  if ((st = status_errors(h))) return bail(st);
  if ((st = evaluate(h, s->w))) return bail(st);
  if ((st = read_status(h))) return bail(st);
  if ((st = status_errors(h))) return bail(st);
  s->f_valid = true;
  *out = s;
  return DP_OK;
}

dp_status dp_system_create_batch(dp_handle* h, int nsys, const int64_t* natoms, const double* x,
                                 const double* v, const int32_t* types,
                                 const double* mass_of_type, const double* boxes,
                                 dp_system** out) {
  CKS(check_handle(h));
  if (!out || !mass_of_type) return fail(h, DP_ERR_ARG, "bad argument");
  *out = nullptr;
  std::unique_ptr<Batch> b(new Batch());
  CKS(batch_init(h, *b, nsys, natoms, boxes));
  const int64_t n = b->base[nsys];
  if (n > 0 && (!x || !v || !types)) return fail(h, DP_ERR_ARG, "null pointer");
  // the system's own fields as dp_system_create sets them (the first box
  // stands in for the batch's: dp_md_step uses the per-system boxes)
  std::vector<double> mass_h(mass_of_type, mass_of_type + h->ntypes_user);
  for (double mm : mass_h)
    if (!(mm > 0)) return fail(h, DP_ERR_ARG, "masses must be > 0");
  std::vector<double> mass_model(DP_MAXT, 0.0), inv_acc(DP_MAXT, 0.0);
  for (int t = 0; t < h->ntypes_user; ++t) {
    const int mt = h->type_map[t];
    if (mass_model[mt] != 0.0 && mass_model[mt] != mass_h[t])
      return fail(h, DP_ERR_UNIMPLEMENTED, "caller types sharing a model type need equal masses");
    mass_model[mt] = mass_h[t];
  }
  for (int t = 0; t < DP_MAXT; ++t) inv_acc[t] = mass_model[t] > 0 ? kAcc / mass_model[t] : 0.0;
  std::unique_ptr<dp_system> s(new dp_system());
  s->h = h;
  if (nsys > 0) std::memcpy(s->box, boxes, sizeof s->box);
  s->mass_user = mass_h;
  if (h->spare_work) {
    s->w = std::move(*h->spare_work);
    h->spare_work.reset();
    s->v = std::move(h->spare_v);
  }
  CKS(load_coords(h, s->w, n, x, types, 0));
  s->types_user.assign(types, types + n);
  CK(ensure(s->v, sizeof(double) * 3 * std::max<int64_t>(n, 1)), "alloc velocities");
  CK(ensure(s->mass, sizeof(double) * DP_MAXT), "alloc masses");
  CK(ensure(s->inv_mass_acc, sizeof(double) * DP_MAXT), "alloc masses");
  if (n) CK(cudaMemcpyAsync(s->v.p, v, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, h->st), "v");
  CK(cudaMemcpyAsync(s->mass.p, mass_model.data(), sizeof(double) * DP_MAXT,
                     cudaMemcpyHostToDevice, h->st),
     "masses");
  CK(cudaMemcpyAsync(s->inv_mass_acc.p, inv_acc.data(), sizeof(double) * DP_MAXT,
                     cudaMemcpyHostToDevice, h->st),
     "masses");
  CKS(clear_status(h));
  CKS(batch_tiles(h, s->w, *b, types));
  CKS(batch_rebuild(h, s->w, *b, h->rc + h->opt.skin));
  CKS(status_errors(h));
  CKS(evaluate_batch(h, s->w, *b));
  CKS(read_status(h));
  CKS(status_errors(h));
  s->batch = std::move(b);
  s->f_valid = true;
  *out = s.release();
  return DP_OK;
}

void dp_system_destroy(dp_system* s) {
  if (!s) return;
  if (s->h && s->h->st) cudaStreamSynchronize(s->h->st);
  if (s->h && !s->h->dead && !s->h->spare_work) {
    // keep the buffers for the handle's next system
    s->h->spare_work.reset(new Work(std::move(s->w)));
    s->h->spare_v = std::move(s->v);
  }
  delete s;
}

int64_t dp_system_step(const dp_system* s) { return s ? s->step : -1; }

int dp_system_batch_size(const dp_system* s) { return s && s->batch ? s->batch->nsys : 0; }

dp_status dp_system_get(dp_system* s, double* x, double* v, double* f, int device_ptrs) {
  if (!s) return DP_ERR_ARG;
  dp_handle* h = s->h;
  CKS(check_handle(h));
  const int64_t n = s->w.n;
  const cudaMemcpyKind kind = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (n) {
    if (x) CK(cudaMemcpyAsync(x, s->w.x.p, sizeof(double) * 3 * n, kind, h->st), "x copy");
    if (v) CK(cudaMemcpyAsync(v, s->v.p, sizeof(double) * 3 * n, kind, h->st), "v copy");
    if (f) CK(cudaMemcpyAsync(f, s->w.f.p, sizeof(double) * 3 * n, kind, h->st), "f copy");
  }
  CK(cudaStreamSynchronize(h->st), "copy");
  return DP_OK;
}

dp_status dp_md_step(dp_handle* h, dp_system* s, int nsteps, double dt_fs, dp_thermo* thermo) {
  CKS(check_handle(h));
  if (!s || s->h != h || nsteps < 0 || !(dt_fs > 0)) return fail(h, DP_ERR_ARG, "bad argument");
  Work& w = s->w;
  const int64_t n = w.n;
  Batch* bt = s->batch.get();  // several systems: their own boxes and lists
  double L[3] = {0.0, 0.0, 0.0};
  if (!bt) CKS(box_lengths(h, s->box, L));
  const double half_skin2 = 0.25 * h->opt.skin * h->opt.skin;
  const double vol = L[0] * L[1] * L[2];
  // one thermo record per step: [KE, PE, virial] of the system, or the
  // per-system sums of batch_seg_launch
  int nvseg = 0;
  if (thermo && bt && n > 0) CKS(batch_seg_upload(h, w, *bt, &nvseg));
  const size_t rec_len = bt ? batch_seg_len(*bt, nvseg, true) : 16;
  if (thermo)
    CK(ensure(s->thermo, sizeof(double) * rec_len * std::max(nsteps, 1)), "alloc thermo");
  CKS(clear_status(h));
  // the launches of a step without a rebuild (kick + drift, FP32 mirror,
  // evaluation, kick); no host synchronisation inside
  auto plain_step = [&]() -> dp_status {
    launch_kick_drift(h->st, n, P<double>(w.x), P<double>(s->v), P<double>(w.f),
                      P<int32_t>(w.types), P<double>(s->inv_mass_acc), dt_fs, P<double>(w.xref),
                      half_skin2, P<int32_t>(h->status));
    if (bt) {
      launch_mirror_batch(h->st, n, P<double>(w.x), P<int32_t>(w.cellc), P<int32_t>(w.types),
                          P<int32_t>(w.sys_of), P<CellGeom>(bt->geoms_dev), P<float4>(w.off));
      CKS(evaluate_batch(h, w, *bt));
    } else {
      launch_mirror(h->st, n, P<double>(w.x), P<int32_t>(w.cellc), P<int32_t>(w.types), w.geom,
                    P<float4>(w.off));
      CKS(evaluate(h, w));
    }
    launch_kick(h->st, n, P<double>(s->v), P<double>(w.f), P<int32_t>(w.types),
                P<double>(s->inv_mass_acc), P<double>(s->mass), dt_fs, nullptr);
    return DP_OK;
  };
  for (int k = 0; k < nsteps; ++k) {
    const bool rebuild_now = (s->step + 1) % h->opt.rebuild_every == 0;
    // graph replay: plain steps, once one plain step since the last rebuild
    // has run normally (every lazy allocation and attribute set is done)
    if (!rebuild_now && h->opt.md_graphs && !h->prof && !thermo && !s->gbroken &&
        s->gplain > 0 && n > 0) {
      if (s->gexec && (s->ggen != g_alloc_gen.load() || s->gdt != dt_fs)) {
        cudaGraphExecDestroy(s->gexec);
        s->gexec = nullptr;
      }
      if (!s->gexec) {
        const unsigned long long l0 = g_dp_launches_tl;
        const unsigned long long gen = g_alloc_gen.load();
        const bool dead0 = h->dead;
        cudaGraph_t graph = nullptr;
        // captured on a private stream (the caller's may be the legacy
        // default stream, which cannot be captured), replayed on the caller's
        if (!h->cap_st) cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking);
        cudaStream_t user_st = h->st;
        bool ok = h->cap_st &&
                  cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        dp_status st = DP_ERR_CUDA;
        if (ok) {
          h->st = h->cap_st;
          st = plain_step();
          h->st = user_st;
          ok = cudaStreamEndCapture(h->cap_st, &graph) == cudaSuccess;
        }
        ok = ok && st == DP_OK && g_alloc_gen.load() == gen;
        if (ok && cudaGraphInstantiate(&s->gexec, graph, 0) != cudaSuccess) {
          s->gexec = nullptr;
          ok = false;
        }
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();  // a failed capture leaves a non-sticky error
        // nothing ran during the capture: a capture error poisons nothing
        h->dead = dead0;
        const unsigned long long nl = g_dp_launches_tl - l0;
        g_dp_launches_tl -= nl;  // counted at each replay instead
        __atomic_fetch_sub(&g_dp_launches, nl, __ATOMIC_RELAXED);
        if (ok) {
          s->ggen = gen;
          s->gdt = dt_fs;
          s->glaunches = nl;
        } else {
          s->gbroken = true;
          h->err.clear();
        }
      }
      if (s->gexec) {
        CK(cudaGraphLaunch(s->gexec, h->st), "graph launch");
        DP_LAUNCHED(s->glaunches);
        s->step += 1;
        s->f_valid = true;
        ++s->gplain;
        continue;
      }
    }
    Phase ph1(h, 4);
    launch_kick_drift(h->st, n, P<double>(w.x), P<double>(s->v), P<double>(w.f),
                      P<int32_t>(w.types), P<double>(s->inv_mass_acc), dt_fs, P<double>(w.xref),
                      half_skin2, P<int32_t>(h->status));
    s->step += 1;
    s->f_valid = false;
    if (s->step % h->opt.rebuild_every == 0) {
      ph1.end();  // the rebuild is timed as its own phase
      CKS(read_status(h));
      CKS(status_errors(h));
      if (bt) CKS(batch_rebuild(h, w, *bt, h->rc + h->opt.skin));
      else CKS(rebuild(h, w, L, h->rc + h->opt.skin));
      // a rebuild may change launch parameters (list capacity, cell grid,
      // tiles) baked into the graph: capture again after it
      s->gplain = 0;
      if (s->gexec) {
        cudaGraphExecDestroy(s->gexec);
        s->gexec = nullptr;
      }
    } else {
      if (bt)
        launch_mirror_batch(h->st, n, P<double>(w.x), P<int32_t>(w.cellc), P<int32_t>(w.types),
                            P<int32_t>(w.sys_of), P<CellGeom>(bt->geoms_dev), P<float4>(w.off));
      else
        launch_mirror(h->st, n, P<double>(w.x), P<int32_t>(w.cellc), P<int32_t>(w.types), w.geom,
                      P<float4>(w.off));
      ++s->gplain;
    }
    ph1.end();
    if (bt) CKS(evaluate_batch(h, w, *bt));
    else CKS(evaluate(h, w));
    Phase ph2(h, 4);
    launch_kick(h->st, n, P<double>(s->v), P<double>(w.f), P<int32_t>(w.types),
                P<double>(s->inv_mass_acc), P<double>(s->mass), dt_fs,
                thermo ? P<double>(w.ke) : nullptr);
    if (thermo && bt) {
      if (n > 0)
        batch_seg_launch(h, w, *bt, nvseg, P<double>(w.ke), P<double>(s->thermo) + rec_len * k);
    } else if (thermo) {
      double* rec = P<double>(s->thermo) + 16 * k;
      launch_sum_rows(h->st, n, 1, P<double>(w.ke), P<double>(w.red_part), rec);
      CK(cudaMemcpyAsync(rec + 1, w.red_out.p, sizeof(double) * 10, cudaMemcpyDeviceToDevice,
                         h->st),
         "thermo");
    }
    s->f_valid = true;
  }
  CK(cudaGetLastError(), "md kernels");
  CKS(read_status(h));
  CKS(status_errors(h));
  if (thermo && bt && nsteps > 0) {
    const int nsys = bt->nsys;
    std::vector<double> rec(rec_len * nsteps, 0.0);
    if (n > 0)
      CK(cudaMemcpy(rec.data(), s->thermo.p, sizeof(double) * rec.size(),
                    cudaMemcpyDeviceToHost),
         "thermo copy");
    for (int k = 0; k < nsteps; ++k) {
      const double* r = rec.data() + rec_len * k;
      for (int q = 0; q < nsys; ++q) {
        dp_thermo& t = thermo[(size_t)k * nsys + q];
        const int64_t dof = 3 * (bt->base[q + 1] - bt->base[q]) - 3;
        const double vq = bt->L[q][0] * bt->L[q][1] * bt->L[q][2];
        t.step = s->step - nsteps + k + 1;
        t.kinetic = r[nsys + 9 * (size_t)nvseg + q] / kAcc;
        t.potential = r[q];
        if (n > 0) batch_seg_virial(*bt, r, q, t.virial);
        else for (int a = 0; a < 9; ++a) t.virial[a] = 0.0;
        t.temperature = dof > 0 ? 2.0 * t.kinetic / (dof * kKb) : 0.0;
        t.pressure =
            (2.0 * t.kinetic + t.virial[0] + t.virial[4] + t.virial[8]) / (3.0 * vq) * kEvA3Bar;
      }
    }
  } else if (thermo && nsteps > 0) {
    std::vector<double> rec((size_t)16 * nsteps);
    CK(cudaMemcpy(rec.data(), s->thermo.p, sizeof(double) * rec.size(), cudaMemcpyDeviceToHost),
       "thermo copy");
    const int64_t dof = 3 * n - 3;
    for (int k = 0; k < nsteps; ++k) {
      const double* r = rec.data() + 16 * k;
      dp_thermo& t = thermo[k];
      t.step = s->step - nsteps + k + 1;
      t.kinetic = r[0] / kAcc;
      t.potential = r[1];
      for (int a = 0; a < 9; ++a) t.virial[a] = r[2 + a];
      t.temperature = dof > 0 ? 2.0 * t.kinetic / (dof * kKb) : 0.0;
      t.pressure = (2.0 * t.kinetic + t.virial[0] + t.virial[4] + t.virial[8]) / (3.0 * vol) * kEvA3Bar;
    }
  }
  return DP_OK;
}

// state file: magic, n, ntypes_user, step, box[9], masses[ntypes_user],
// types[n], x[n][3], v[n][3], f[n][3], xref[n][3]
dp_status dp_state_save(dp_system* s, const char* path) {
  if (!s || !path) return DP_ERR_ARG;
  dp_handle* h = s->h;
  CKS(check_handle(h));
  const int64_t n = s->w.n;
  const Batch* bt = s->batch.get();
  std::vector<double> x(3 * n), v(3 * n), f(3 * n), xr(3 * n);
  if (n) {
    CK(cudaStreamSynchronize(h->st), "sync");
    CK(cudaMemcpy(x.data(), s->w.x.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost), "copy");
    CK(cudaMemcpy(v.data(), s->v.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost), "copy");
    CK(cudaMemcpy(f.data(), s->w.f.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost), "copy");
    CK(cudaMemcpy(xr.data(), s->w.xref.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost), "copy");
  }
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return fail(h, DP_ERR_ARG, "cannot open state file for writing");
  int64_t hdr[3] = {n, (int64_t)s->mass_user.size(), s->step};
  bool ok;
  if (bt) {
    // several systems: their count, atom counts and boxes after the header
    const int64_t nsys = bt->nsys;
    std::vector<int64_t> counts(nsys);
    for (int q = 0; q < bt->nsys; ++q) counts[q] = bt->base[q + 1] - bt->base[q];
    ok = std::fwrite("DPSTATE2", 1, 8, fp) == 8 && std::fwrite(hdr, 8, 3, fp) == 3 &&
         std::fwrite(&nsys, 8, 1, fp) == 1 &&
         std::fwrite(counts.data(), 8, counts.size(), fp) == counts.size() &&
         std::fwrite(bt->boxes.data(), 8, bt->boxes.size(), fp) == bt->boxes.size();
  } else {
    ok = std::fwrite("DPSTATE1", 1, 8, fp) == 8 && std::fwrite(hdr, 8, 3, fp) == 3 &&
         std::fwrite(s->box, 8, 9, fp) == 9;
  }
  ok = ok &&
            std::fwrite(s->mass_user.data(), 8, s->mass_user.size(), fp) == s->mass_user.size() &&
            std::fwrite(s->types_user.data(), 4, n, fp) == (size_t)n &&
            std::fwrite(x.data(), 8, 3 * n, fp) == (size_t)(3 * n) &&
            std::fwrite(v.data(), 8, 3 * n, fp) == (size_t)(3 * n) &&
            std::fwrite(f.data(), 8, 3 * n, fp) == (size_t)(3 * n) &&
            std::fwrite(xr.data(), 8, 3 * n, fp) == (size_t)(3 * n);
  std::fclose(fp);
  return ok ? DP_OK : fail(h, DP_ERR_ARG, "state write failed");
}

dp_status dp_state_load(dp_handle* h, const char* path, dp_system** out) {
  CKS(check_handle(h));
  if (!path || !out) return fail(h, DP_ERR_ARG, "bad argument");
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return fail(h, DP_ERR_ARG, "cannot open state file");
  char magic[8];
  int64_t hdr[3];
  double box[9];
  bool ok = std::fread(magic, 1, 8, fp) == 8;
  const bool several = ok && std::memcmp(magic, "DPSTATE2", 8) == 0;
  ok = ok && (several || std::memcmp(magic, "DPSTATE1", 8) == 0) &&
       std::fread(hdr, 8, 3, fp) == 3 && hdr[0] >= 0 && hdr[0] < (1LL << 31) &&
       hdr[1] == h->ntypes_user;
  // several systems: their count, atom counts (summing to n) and boxes
  int64_t nsys = 0;
  std::vector<int64_t> counts;
  std::vector<double> boxes;
  if (ok && several) {
    ok = std::fread(&nsys, 8, 1, fp) == 1 && nsys >= 0 && nsys < (1 << 24);
    if (ok) {
      counts.resize(nsys);
      boxes.resize(9 * (size_t)nsys);
      ok = std::fread(counts.data(), 8, nsys, fp) == (size_t)nsys &&
           std::fread(boxes.data(), 8, boxes.size(), fp) == boxes.size();
      int64_t tot = 0;
      for (int64_t c : counts) {
        ok = ok && c >= 0;
        tot += c;
      }
      ok = ok && tot == hdr[0];
    }
  } else if (ok) {
    ok = std::fread(box, 8, 9, fp) == 9;
  }
  const int64_t n = ok ? hdr[0] : 0;
  std::vector<double> mass(ok ? hdr[1] : 0), x(3 * n), v(3 * n), f(3 * n), xr(3 * n);
  std::vector<int32_t> types(n);
  ok = ok && std::fread(mass.data(), 8, mass.size(), fp) == mass.size() &&
       std::fread(types.data(), 4, n, fp) == (size_t)n &&
       std::fread(x.data(), 8, 3 * n, fp) == (size_t)(3 * n) &&
       std::fread(v.data(), 8, 3 * n, fp) == (size_t)(3 * n) &&
       std::fread(f.data(), 8, 3 * n, fp) == (size_t)(3 * n) &&
       std::fread(xr.data(), 8, 3 * n, fp) == (size_t)(3 * n);
  std::fclose(fp);
  if (!ok) return fail(h, DP_ERR_ARG, "malformed state file");
  // rebuild the list from the reference positions of the saved list, then
  // restore the current positions and forces: the continued run then sees
  // the same list, cells and forces as the run that was saved
  dp_system* s = nullptr;
  if (several)
    CKS(dp_system_create_batch(h, (int)nsys, counts.data(), xr.data(), v.data(), types.data(),
                               mass.data(), boxes.data(), &s));
  else
    CKS(dp_system_create(h, n, xr.data(), v.data(), types.data(), mass.data(), box, 0, &s));
  s->step = hdr[2];
  if (n) {
    if (cudaMemcpy(s->w.x.p, x.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice) ||
        cudaMemcpy(s->w.f.p, f.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice)) {
      dp_system_destroy(s);
      return fail(h, DP_ERR_CUDA, "state upload failed");
    }
    if (s->batch)
      launch_mirror_batch(h->st, n, P<double>(s->w.x), P<int32_t>(s->w.cellc),
                          P<int32_t>(s->w.types), P<int32_t>(s->w.sys_of),
                          P<CellGeom>(s->batch->geoms_dev), P<float4>(s->w.off));
    else
      launch_mirror(h->st, n, P<double>(s->w.x), P<int32_t>(s->w.cellc),
                    P<int32_t>(s->w.types), s->w.geom, P<float4>(s->w.off));
  }
  s->f_valid = true;
  *out = s;
  return DP_OK;
}

}  // extern "C"
