/*
 * dp.h -- C ABI of the GB300 compressed Deep Potential (DP-SE_a) library.
 *
 * The library evaluates the energy, forces and virial of the DP-SE_a model of
 * arXiv 2201.01446 with the embedding net replaced by the paper's fifth-order
 * piecewise-polynomial table (Sec. 3.2) fused with the R^T G contraction
 * (Sec. 3.4.1), and integrates velocity-Verlet molecular dynamics (Sec. 4).
 * Every step runs in the library's own CUDA kernels for sm_103a.
 *
 * Conventions for every call:
 *   - Units: energy eV, length A, time fs, mass amu, force eV/A, virial eV.
 *   - Arrays are row-major.  coords/forces/velocities are [natoms][3].
 *     box is [3][3] with the cell vectors as rows; only orthorhombic boxes
 *     (off-diagonal entries exactly 0) are accepted, else DP_ERR_BOX.
 *   - Ownership: the caller owns every array it passes.  Inputs are copied
 *     (host pointers) or read in place on the handle's stream (device
 *     pointers); the library never frees or keeps caller memory.  The handle
 *     owns every device buffer it allocates.
 *   - Errors: each call returns a dp_status and never aborts.  On error the
 *     outputs are unspecified and the handle stays usable, except after
 *     DP_ERR_CUDA, which is sticky (destroy the handle).  dp_last_error()
 *     gives a one-line message.
 *   - Threads: a handle (and the systems made from it) belongs to one host
 *     thread at a time.  All device work is ordered on the handle's stream.
 */
#ifndef DP_GB300_H
#define DP_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DP_OK = 0,
  DP_ERR_ARG = 1,           /* bad argument (NULL, negative size, bad type index) */
  DP_ERR_MODEL = 2,         /* model file missing or malformed */
  DP_ERR_CUDA = 3,          /* CUDA runtime/kernel failure (sticky) */
  DP_ERR_OOM = 4,           /* device allocation failed */
  DP_ERR_SEL_OVERFLOW = 5,  /* more neighbors of one type within rc than sel[t] */
  DP_ERR_TABLE_RANGE = 6,   /* an s(r) beyond the table's last node */
  DP_ERR_BOX = 7,           /* box not orthorhombic, or an edge shorter than the list cutoff */
  DP_ERR_TIMEOUT = 8,       /* a bounded wait gave up */
  DP_ERR_UNIMPLEMENTED = 9, /* option combination not built */
  DP_ERR_SKIN = 10,         /* an atom moved more than skin/2 between list rebuilds */
  DP_ERR_NONFINITE = 11,    /* a non-finite energy or force was produced */
  DP_ERR_CAPACITY = 12      /* request larger than a fixed capacity (see below) */
} dp_status;

typedef struct dp_handle dp_handle;
typedef struct dp_system dp_system;

/* Evaluation options.  dp_options_default() fills the defaults in brackets. */
typedef struct {
  int tabulated;       /* 1: tabulated embedding fused with the contraction
                          (Sec. 3.2-3.4) [1]; 0: plain untabulated FP32 net */
  int fit_precision;   /* fitting-net GEMMs: 0 FP32 CUDA cores [0],
                          1 BF16 tcgen05 tensor cores with FP32 accumulation,
                          2 FP32-accurate tcgen05: each operand three BF16
                          pieces x = h + m + l (six piece products per
                          multiply-add),
                          3 near-FP32 tcgen05: each operand an FP16 pair
                          x s = h + l, s a power of two from a bound of |x|
                          (three piece products; errors about 1.5x those of
                          mode 2, stated, not bound to the FP32 bars),
                          4 mode 2 with the dE/dD GEMM (Eq. 2's input
                          gradient, forces only) on FP16 pairs */
  double table_step;   /* interval h of the table on s (Sec. 3.2) [0.01] */
  double s_max;        /* table domain is [0, ceil(s_max/h)*h]; [2.0], i.e.
                          r >= 0.5 A for rcs = 0.5 */
  double skin;         /* neighbor-list buffer for MD (Sec. 4) [2.0 A] */
  int rebuild_every;   /* MD list rebuild period in steps [10] */
  int embed_precision; /* tabulated embedding contraction: 0 FP32 CUDA cores
                          [0], 2 FP32-accurate tcgen05 tensor cores (split
                          operands); the plain path ignores it */
  int tanh_table;      /* fitting-net activation: 0 tanh [0]; 1 the tanh table
                          of Sec. 3.5 (second order on [0, 8) in intervals of
                          1/128, odd, 1 beyond 8; error < 2.3e-7) */
  int md_graphs;       /* dp_md_step: 1 [1] replays the launches of a step
                          without a list rebuild as one CUDA graph (captured
                          once per system and invalidated when a buffer is
                          reallocated); 0 launches every kernel.  The results
                          are bitwise the same; not used while profiling or
                          when thermo output is requested */
  double s_ext;        /* table extrapolation region: beyond the first region
                          [0, n_fine*h], n_fine = ceil(s_max/h), intervals of
                          width ext_stride*h up to the first node >= s_ext;
                          [0.0] none (s_ext <= n_fine*h); negative is
                          DP_ERR_ARG */
  int ext_stride;      /* width of the extrapolation intervals in units of h,
                          1 .. 1000 (DP_ERR_ARG otherwise) [10] */
} dp_options;

/* Thermodynamic record of one MD step (Sec. 4). */
typedef struct {
  int64_t step;
  double kinetic;     /* eV */
  double potential;   /* eV */
  double temperature; /* K, 3N-3 degrees of freedom */
  double pressure;    /* bar, (2 KE + tr(virial)) / (3 V) */
  double virial[9];   /* eV */
} dp_thermo;

void dp_options_default(dp_options* opt);

/*
 * dp_create -- load a model, build its table on the device, bind a stream.
 *   model_path  DPSEAV01 model file (embedding nets per (centre, neighbor)
 *               type pair, fitting net per centre type; Sec. 2.1, Eq. 3-5).
 *   ntypes      number of atom types the caller will use (<= 8).
 *   type_map    [ntypes] model type of each caller type, or NULL (identity).
 *   rc, rcs     cutoff radius and start of the smooth switch (Eq. 1), A.
 *   sel         [model ntypes] maximum neighbors of each type within rc; the
 *               N_m of Eq. 2 is their sum.
 *   opt         options or NULL for the defaults.
 *   stream      cudaStream_t to order all work on, or NULL (legacy default).
 *   out         receives the handle.
 * Errors: DP_ERR_ARG, DP_ERR_MODEL, DP_ERR_OOM, DP_ERR_CUDA.
 */
dp_status dp_create(const char* model_path, int ntypes, const int32_t* type_map, double rc,
                    double rcs, const int32_t* sel, const dp_options* opt, void* stream,
                    dp_handle** out);

/* Destroy a handle and free its device memory.  NULL is a no-op. */
void dp_destroy(dp_handle* h);

/* Last error message of the handle (never NULL; "" after success).  With
 * h == NULL: the message of the last failed dp_create on this thread. */
const char* dp_last_error(const dp_handle* h);

/* Change the stream the handle orders its work on (cudaStream_t). */
dp_status dp_set_stream(dp_handle* h, void* stream);

/*
 * dp_compute -- one energy/force/virial evaluation (Sec. 2.1):
 *   E = sum_i E_i,  F_i = -dE/dr_i,  virial = -sum_ij r_ij (x) dE_i/dr_ij.
 *   natoms      >= 0.  coords [natoms][3] (A, need not be wrapped),
 *   types       [natoms] caller types, box [3][3].
 *   device_ptrs 0: all array arguments are host memory (the call copies in
 *               and out and returns after the results are on the host);
 *               1: all are device memory (the call is asynchronous on the
 *               handle's stream except for the status check at its end).
 *   energy      [1] eV; forces [natoms][3]; virial [9] (row-major, symmetric);
 *   atom_energy [natoms] or NULL.
 * The neighbor list is built fresh with cutoff rc.
 * Errors: DP_ERR_ARG, DP_ERR_BOX, DP_ERR_SEL_OVERFLOW, DP_ERR_TABLE_RANGE,
 *         DP_ERR_NONFINITE, DP_ERR_OOM, DP_ERR_CUDA.
 */
dp_status dp_compute(dp_handle* h, int64_t natoms, const double* coords, const int32_t* types,
                     const double* box, int device_ptrs, double* energy, double* forces,
                     double* virial, double* atom_energy);

/*
 * dp_system_create -- a device-resident MD system (positions, velocities,
 * forces in FP64; neighbor list with skin; CUDA graph of the step block).
 *   x, v [natoms][3] (A, A/fs), types [natoms], mass_of_type [ntypes] (amu),
 *   box [3][3]; device_ptrs as in dp_compute.  Copies everything in.
 */
dp_status dp_system_create(dp_handle* h, int64_t natoms, const double* x, const double* v,
                           const int32_t* types, const double* mass_of_type, const double* box,
                           int device_ptrs, dp_system** out);
/* Several independent systems as one MD system (a serving batch of small MD
 * requests): natoms [nsys], x, v [sum natoms][3] and types [sum natoms] the
 * systems one after another, boxes [nsys][3][3], mass_of_type as above (HOST
 * arrays).  dp_md_step then advances all of them (one launch of each kernel;
 * each system keeps its own box, cells and neighbor list, rebuilt on the
 * common schedule), dp_system_get returns the concatenated arrays.  Each
 * system's trajectory is bitwise the one it has alone, and so are its thermo
 * records (dp_md_step writes [nsteps][nsys] of them); dp_state_save and
 * dp_state_load keep all the systems.  Needs tabulated = 1 and
 * embed_precision = 2. */
dp_status dp_system_create_batch(dp_handle* h, int nsys, const int64_t* natoms, const double* x,
                                 const double* v, const int32_t* types,
                                 const double* mass_of_type, const double* boxes,
                                 dp_system** out);
/* Frees the system.  The handle keeps the device buffers of the last
 * destroyed system (lists, T, dT, sorted pairs ...) and gives them to its
 * next dp_system_create, so a stream of systems does not allocate and free
 * gigabytes each time; dp_destroy releases them.  Destroy every system
 * before its handle. */
void dp_system_destroy(dp_system* s);

/* Copy x, v, f (any may be NULL) out of the system; device_ptrs as above.
 * Positions come back wrapped into the box as of the last list rebuild. */
dp_status dp_system_get(dp_system* s, double* x, double* v, double* f, int device_ptrs);

/* Current step count of the system. */
int64_t dp_system_step(const dp_system* s);

/* Number of systems of a system made by dp_system_create_batch; 0 for one
 * made by dp_system_create or dp_state_load. */
int dp_system_batch_size(const dp_system* s);

/*
 * dp_md_step -- nsteps velocity-Verlet steps of dt_fs (Sec. 4):
 *   v += dt/2 F/m;  x += dt v;  (list rebuild when step % rebuild_every == 0);
 *   F = -grad E;  v += dt/2 F/m.
 * The rebuild schedule is keyed to the absolute step count, so a run split
 * into several calls (or saved and loaded) follows the same schedule.
 * thermo_out: NULL, or [nsteps] records (one per step, after the step);
 *   for a batch system [nsteps][nsys], one per system (its own atoms, 3N-3
 *   degrees of freedom, box volume and virial).
 * Errors: as dp_compute, plus DP_ERR_SKIN.
 */
dp_status dp_md_step(dp_handle* h, dp_system* s, int nsteps, double dt_fs, dp_thermo* thermo_out);

/* Save / load the MD state (x, v, f, types, masses, box, step and the
 * list's reference positions) to a file; a batch system's file holds every
 * system (atom counts and boxes) and loads as a batch system.  A loaded
 * system continues bitwise as the saved one would have. */
dp_status dp_state_save(dp_system* s, const char* path);
dp_status dp_state_load(dp_handle* h, const char* path, dp_system** out);

/* ---------------------------------------------------------------------------
 * Inspection calls used by the parity tests.
 * ------------------------------------------------------------------------- */

/* Neighbor pairs with |r_ij| < rlist as rows (i, j, n0, n1, n2), where n is the
 * periodic image: r_ij = x_j + n*L - x_i with x wrapped into [0, L).  Host
 * arrays.  Writes at most cap rows (in the library's list order, not sorted)
 * and returns the total count in *count. */
dp_status dp_neighbor_pairs(dp_handle* h, int64_t natoms, const double* coords,
                            const double* box, double rlist, int64_t cap, int32_t* out5,
                            int64_t* count);

/* The device table of model type pair (ti, tj) as FP32 [n][6][M]: on
 * interval k, [x_k, x_k + w_k), the embedding row is sum_q c[k][q][:] u^q
 * with the normalised local variable u = (s - x_k)/w_k in [0, 1), i.e.
 * c[k][q] = a_q w_k^q for the paper's coefficients a_q of the local variable
 * s - x_k (Sec. 3.2).  x_k = k h and w_k = h in the first region (k <
 * n_fine); beyond it w_k = ext_stride*h (see dp_options.s_ext).
 * *n receives the interval count (call with out == NULL to query it). */
dp_status dp_table_coeffs(dp_handle* h, int ti, int tj, float* out, int32_t* n);

/* Per-atom T = R^T G / N_m, FP32 [natoms][4][M] (host arrays). */
dp_status dp_descriptor(dp_handle* h, int64_t natoms, const double* coords,
                        const int32_t* types, const double* box, float* T_out);

/* The descriptor and fitting stage alone (Eq. 2, Sec. 2.1) in the handle's
 * fit_precision: per-atom energies E_i and dE_i/dT for given T.
 *   types  HOST [natoms] caller types; T HOST FP32 [natoms][4][M];
 *   e_out  HOST [natoms] eV; dT_out HOST FP32 [natoms][4][M] or NULL. */
dp_status dp_fitting(dp_handle* h, int64_t natoms, const int32_t* types, const float* T,
                     double* e_out, float* dT_out);

/* Several independent systems in one evaluation (a serving batch of small
 * boxes): one neighbor list per system, one launch of each embedding and
 * fitting kernel over all atoms.  HOST arrays:
 *   natoms  [nsys] atoms per system; coords [sum natoms][3] and types
 *           [sum natoms], the systems one after another;
 *   boxes   [nsys][3][3] orthorhombic boxes (rows);
 *   energies [nsys] eV; forces [sum natoms][3] eV/A; virials [nsys][9] eV.
 * Needs tabulated = 1 and embed_precision = 2 (DP_ERR_UNIMPLEMENTED
 * otherwise).  A system's energy, forces and virial are bitwise those of
 * dp_compute on it alone (its atoms are grouped in the same tiles of 32 and
 * every sum runs in the same order).  An error in any system (sel
 * overflow, table range, box) fails the call. */
dp_status dp_compute_batch(dp_handle* h, int nsys, const int64_t* natoms, const double* coords,
                           const int32_t* types, const double* boxes, double* energies,
                           double* forces, double* virials);

/* ---------------------------------------------------------------------------
 * Parameter gradients (training use of the same energy, Sec. 2.1 and 3.2):
 * dE/d(fitting-net parameters) and dE/d(table coefficients).
 *
 * Fitting layout, per model type in type order, per hidden layer k a block of
 * [(win_k + 1)][wout_k] doubles (W_k row-major, then b_k), then [(w_last + 1)]
 * (w_out, then b_out).  The embedding representation ("table" arrays): for
 * a tabulated handle the table, [ntypes][ntypes][n][6][M] in the layout of
 * dp_table_coeffs (the derivative with respect to c[k][q][:], the
 * coefficient of u^q with u = (s - x_k)/w_k); for an untabulated handle
 * (tabulated = 0) the embedding nets' weights and biases, per (centre,
 * neighbor) type pair per layer a [(win_k + 1)][wout_k] block, win_0 = 1.
 * ------------------------------------------------------------------------- */
/* *n_fit: doubles of the fitting gradient (all types); *n_table: doubles of
 * the table gradient.  Either pointer may be NULL. */
dp_status dp_param_sizes(dp_handle* h, int64_t* n_fit, int64_t* n_table);

/* Energy and its parameter gradients for one configuration (HOST arrays,
 * the conventions of dp_compute).  The fitting stage runs on the FP32 CUDA
 * cores whatever fit_precision says; the gradients are summed per chunk in
 * FP32 and across chunks in FP64 (deterministic).
 *   grad_fit   HOST [n_fit] (required, overwritten);
 *   grad_table HOST [n_table] or NULL.  A tabulated handle needs
 *              embed_precision = 2 (DP_ERR_UNIMPLEMENTED otherwise).
 * Errors as dp_compute (DP_ERR_SEL_OVERFLOW, DP_ERR_TABLE_RANGE, ...). */
dp_status dp_param_grad(dp_handle* h, int64_t natoms, const double* coords,
                        const int32_t* types, const double* box, double* energy,
                        double* grad_fit, double* grad_table);

/* The model's current parameters in the same two layouts (HOST arrays of
 * n_fit and n_table doubles; either may be NULL).  The device keeps FP32
 * copies of the fitting nets and the table, so those come back as FP32
 * values; an untabulated handle's embedding nets come back as loaded. */
dp_status dp_get_params(dp_handle* h, double* fit, double* table);

/* Replace the fitting parameters and/or the embedding representation
 * (either pointer may be NULL), e.g. after a gradient step, in the layouts of
 * dp_param_grad: the table coefficients of a tabulated handle, the embedding
 * nets' weights and biases of an untabulated one.  Values are rounded to FP32
 * for the device copies and every derived copy (transposes, BF16 pieces,
 * tiled table operands; for new embedding nets the FP32 nets and the
 * handle's table, which dp_table_coeffs then returns) is rebuilt.
 * Synchronous. */
dp_status dp_set_params(dp_handle* h, const double* fit, const double* table);

/* ---------------------------------------------------------------------------
 * Profiling: per-phase device time measured with CUDA events recorded on the
 * handle's stream around each phase's kernels.
 * ------------------------------------------------------------------------- */
#define DP_NPHASE 5
/* phases: 0 neighbor-list build (cell binning, lists), 1 environment matrix +
 * tabulated embedding + contraction (forward), 2 descriptor + fitting net
 * forward and backward, 3 tabulated contraction backward + forces + virial,
 * 4 integration, force finalisation and reductions */

/* enable = 1: reset and start recording; 0: stop. */
dp_status dp_profile(dp_handle* h, int enable);
/* ms[DP_NPHASE]: summed device time per phase since the last reset;
 * launches[DP_NPHASE]: number of timed phase executions.  Synchronises the
 * handle's stream. */
dp_status dp_profile_read(dp_handle* h, double* ms, int64_t* launches);

/* Counters of the last evaluation of a system (s != NULL) or of the last
 * dp_compute (s == NULL): out[0] atoms, [1] list capacity per atom, [2]
 * longest list, [3] pairs within rc seen by the last forward pass, [4] cells,
 * [5] kernels launched by the library in this process so far. */
dp_status dp_stats(dp_handle* h, const dp_system* s, int64_t* out);

/*
 * dp_neighbor_pairs_static -- the pair rows of dp_neighbor_pairs, computed
 * without allocating any memory.  For callers that must not call cudaMalloc
 * or cudaFree: an MD engine that owns all device memory through its own
 * pool, or a time-critical loop where an allocation (which can synchronise
 * the whole device) is not acceptable.  The paper has no counterpart; it
 * is a service of this library.
 *   natoms      0 <= natoms <= 65536, else DP_ERR_CAPACITY.
 *   coords      DEVICE [natoms][3] positions (A), need not be wrapped.
 *   box         HOST [3][3] orthorhombic box; rlist <= every edge and at
 *               most 65536 cells of edge >= rlist (else DP_ERR_BOX /
 *               DP_ERR_CAPACITY).
 *   cap, out5   DEVICE [cap][5] int32 rows (i, j, n0, n1, n2) as in
 *               dp_neighbor_pairs; rows past cap are not written.
 *   count       HOST: receives the total number of pairs (64-bit; it
 *               may exceed 2^31, e.g. for a box of edge close to rlist).
 *   stream      cudaStream_t (NULL = legacy default); the call returns after
 *               the stream has finished its work.
 * All intermediates live in one fixed device array of about 5 MB that every
 * GPU loading the library keeps until the process exits.  Calls share it:
 * calls whose device work overlaps (other streams or host threads without
 * ordering) race.  The first call on a device looks up the array's device
 * address with that device current; make it before any stream capture.
 */
dp_status dp_neighbor_pairs_static(int64_t natoms, const double* coords, const double* box,
                                   double rlist, int64_t cap, int32_t* out5, int64_t* count,
                                   void* stream);

/* Device memory held by the library (every buffer it allocated with
 * cudaMalloc and has not freed).  Any pointer may be NULL.
 *   handle_bytes   bytes held by the handle h (model, tables, work areas,
 *                  scratch, buffers kept from destroyed systems; not those
 *                  of live systems); needs h != NULL (else DP_ERR_ARG).
 *   process_bytes  bytes held by all handles and systems of the process.
 *   process_peak   the most process_bytes has been since the last reset.
 *   reset_peak     non-zero: restart the peak at the current value.
 * Host-side counters: no device work, no synchronisation. */
dp_status dp_memory(const dp_handle* h, int64_t* handle_bytes, int64_t* process_bytes,
                    int64_t* process_peak, int reset_peak);

/* Release the handle's work area, the buffers kept from its destroyed
 * systems and its fitting / gradient scratch (all are allocated again on
 * demand, so a memory budget can reclaim an idle handle's cache).  The model,
 * tables and live systems stay.  Synchronises the handle's stream. */
dp_status dp_trim(dp_handle* h);

/* FP32 FMA throughput probe (measurement only; the paper has no
 * counterpart): one launch on `stream` of a kernel in which every resident
 * thread of every SM runs independent FMA chains, `outer` x 512 FMAs per
 * thread; *flops receives the FLOPs it performs (2 per FMA).  Timing the
 * launch with CUDA events on that stream gives the FP32 CUDA-core peak at the
 * clock the GPU runs at.  Errors: DP_ERR_ARG (outer < 1, flops NULL),
 * DP_ERR_CUDA. */
dp_status dp_fma_peak_run(int64_t outer, void* stream, double* flops);

/* Library build string (architecture, options compiled in). */
const char* dp_version(void);

#ifdef __cplusplus
}
#endif
#endif
