/*
 * FP64 CPU oracle for the compressed DP-SE_a energy / force / virial path.
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the correctness reference that the
 * CUDA path is checked against; it is never part of the product path.  It
 * shares no code, header, table or constant with the CUDA library: the only
 * thing both sides read is the model file written by the seeded generator.
 *
 * Every function follows the paper (arXiv 2201.01446, Sec. 2 and Sec. 3.2):
 *   Eq. 1   environment matrix rows s(r) * (1, x/r, y/r, z/r)
 *   Eq. 2   descriptor D = (G^<)^T R R^T G
 *   Eq. 3-5 embedding net, tanh first layer, (x,x)+tanh(xW+b) later layers
 *   Sec. 2.1 fitting net with shortcuts, E = sum_i E_i, F = -grad E
 *   Sec. 3.2 fifth-order piecewise polynomial table matching value, first
 *            and second derivative at the interval nodes
 *   Sec. 4   velocity-Verlet MD
 * Readings of passages the paper leaves open (switch function, 1/N_m
 * scaling, descriptor flattening order, virial sign, local polynomial
 * variable) are stated beside the code that takes them.
 *
 * All arrays are caller-owned, row-major, float64 unless stated.
 */
#ifndef DP_ORACLE_H
#define DP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_OK = 0,
  ORC_ERR_ARG = 1,
  ORC_ERR_MODEL = 2,
  ORC_ERR_NOMEM = 4,
  ORC_ERR_SEL = 5,
  ORC_ERR_TABLE_RANGE = 6,
  ORC_ERR_BOX = 7
};

typedef struct orc_model orc_model;
typedef struct orc_table orc_table;

void orc_set_threads(int nthreads);
int orc_get_threads(void);

/* model file (format documented in the generator module) */
orc_model* orc_model_load(const char* path);
void orc_model_free(orc_model* m);
/* dims[0..5] = ntypes, M, m_lt, din, emb_w[0], n_fit */
int orc_model_dims(const orc_model* m, int32_t* dims);

/* smooth switch (reading of Eq. 1's gate): sw=1 for r<rcs, quintic
 * 1-10u^3+15u^4-6u^5 for rcs<=r<rc with u=(r-rcs)/(rc-rcs), 0 for r>=rc. */
void orc_switch(double r, double rc, double rcs, double* sw, double* dsw);
/* Eq. 1 row for displacement d=r_ij: R[4] and dR[4][3] = dR_c/dd_beta; returns s */
double orc_env_row(const double* d, double rc, double rcs, double* R, double* dR);

/* Eq. 3-5: G row g(s) of the (ti,tj) embedding net with exact first and
 * second derivative in s (forward-mode).  dg / d2g may be NULL. */
int orc_embed(const orc_model* m, int ti, int tj, double s, double* g, double* dg, double* d2g);

/* Sec. 3.5 tanh table for the fitting net (off by default): second order on
 * [0, 8) with step 1/128, odd, 1 beyond 8; orc_act is the activation the
 * fitting net uses (dt: its derivative) */
void orc_set_tanh_table(int on);
double orc_act(double a, double* dt);

/* fitting net of centre type ti: E(D); dD (length din) = dE/dD if not NULL */
int orc_fit(const orc_model* m, int ti, const double* D, double* E, double* dD);

/* Sec. 3.2 tabulation: nodes x_k = k*h, k=0..n with n=ceil(s_max/h) */
orc_table* orc_table_build(const orc_model* m, double h, double s_max);
/* The same with an extrapolation region: intervals of width h up to
 * n_fine h >= s_max, then of width stride*h up to the first node >= s_ext
 * (none when s_ext <= n_fine h).  Each interval is the quintic matching the
 * net's value and first two derivatives at its two nodes (Sec. 3.2); the
 * coarser second region is an extension of the paper's equal division. */
orc_table* orc_table_build_ext(const orc_model* m, double h, double s_max, double s_ext,
                               int stride);
/* the extrapolation layout: intervals of width h, width of the others */
int orc_table_ext(const orc_table* t, int32_t* n_fine, double* H);
void orc_table_free(orc_table* t);
int orc_table_dims(const orc_table* t, int32_t* n, double* h);
/* coefficients of pair (ti,tj): out[n][6][M], local variable t = s - x_k
 * (x_k = k h in the first region) */
int orc_table_coeffs(const orc_table* t, int ti, int tj, double* out);
/* evaluate the table: g[M], dg[M]; returns 1 when s is beyond the last node */
int orc_table_eval(const orc_table* t, int ti, int tj, double s, double* g, double* dg);
/* quintic on [0,h] matching (y,y',y'') at both ends: a[0..5] */
void orc_hermite5(const double* y0, const double* y1, double h, double* a);

/* periodic wrap used by both neighbor builders: x - L*floor(x/L) into [0,L) */
double orc_wrap(double x, double L);

/* neighbor pairs (i, j, n0, n1, n2) with |x_j + n*L - x_i| < rlist (wrapped
 * x), (j,n) != (i,0).  method 0 = brute force over images, 1 = cell list.
 * Writes at most cap rows into out5 (sorted by i, j, n) and returns the
 * total count, or -errcode. */
int64_t orc_neighbors(int64_t n, const double* x, const double* box, double rlist,
                      int method, int64_t cap, int32_t* out5);

/* Full evaluation.  table == NULL selects the original embedding net.
 * atom_energy may be NULL.  diag (may be NULL) receives
 * [0]=max neighbor count over atoms, [1]=pairs within rc, [2]=table range
 * violations, [3]=atoms whose per-type count exceeded sel. */
int orc_eval(const orc_model* m, const orc_table* table, double rc, double rcs,
             const int32_t* sel, int64_t n, const double* x, const int32_t* types,
             const double* box, double* energy, double* atom_energy, double* force,
             double* virial, int64_t* diag);

/* Per-atom pieces for atom i: T[4][M] (with the 1/N_m factor) and D[M*m_lt]. */
int orc_atom_descriptor(const orc_model* m, const orc_table* table, double rc, double rcs,
                        const int32_t* sel, int64_t n, const double* x, const int32_t* types,
                        const double* box, int64_t i, double* T, double* D);

/* Sampled evaluation of a large system: E_i for the atoms idx_e[0..ne) and
 * the forces on the atoms idx_f[0..nf) (computed from every centre within rc). */
int orc_eval_subset(const orc_model* m, const orc_table* table, double rc, double rcs,
                    const int32_t* sel, int64_t n, const double* x, const int32_t* types,
                    const double* box, int64_t ne, const int64_t* idx_e, double* e_out,
                    int64_t nf, const int64_t* idx_f, double* f_out);

/* Velocity-Verlet NVE (Sec. 4): nsteps steps of dt fs.  x, v (A, A/fs) are
 * updated in place; f receives the final forces.  With f_valid != 0, f on
 * entry already holds the forces at x and the initial evaluation is skipped.
 * thermo (may be NULL) receives (nsteps+1) rows of (KE eV, PE eV, T K, P bar)
 * (row 0 has PE = 0 and a kinetic-only pressure when f_valid != 0). */
int orc_md(const orc_model* m, const orc_table* table, double rc, double rcs,
           const int32_t* sel, int64_t n, double* x, double* v, double* f, int f_valid,
           const int32_t* types, const double* mass_of_type, const double* box,
           double dt, int nsteps, double* thermo);

/* Parameter gradients of the same energy.  Per centre type the fitting
 * parameters are laid out as one [(win_k + 1)][wout_k] block per layer k
 * (W_k rows, then b_k) followed by [(w_last + 1)] (w_out, then b_out);
 * orc_fit_param_count gives the length of one type's layout. */
int64_t orc_fit_param_count(const orc_model* m);
/* copy type ti's fitting parameters out (get) and/or replace them (set) */
int orc_model_fit_params(orc_model* m, int ti, double* get, const double* set);
/* replace the coefficients of pair (ti,tj) ([n][6][M], local variable s - k*h) */
int orc_table_set_coeffs(orc_table* t, int ti, int tj, const double* in);
/* per (centre, neighbor) type pair: the embedding net's parameters, layer k
 * as a [(win_k + 1)][wout_k] block (W_k rows, then b_k), win_0 = 1 */
int64_t orc_emb_param_count(const orc_model* m);
int orc_model_emb_params(orc_model* m, int ti, int tj, double* get, const double* set);
/* energy and dE/d(fitting parameters) of all centre types (grad_fit:
 * ntypes x orc_fit_param_count) and dE/d(embedding representation) in
 * grad_table (may be NULL): for a tabulated model the table coefficients
 * [ntypes*ntypes][n][6][M] with respect to c_q = a_q h^q, the coefficients of
 * the normalised local variable (s - k*h)/h; for the original net
 * (table == NULL) its weights and biases [ntypes*ntypes][orc_emb_param_count] */
int orc_param_grad(const orc_model* m, const orc_table* table, double rc, double rcs,
                   const int32_t* sel, int64_t n, const double* x, const int32_t* types,
                   const double* box, double* energy, double* grad_fit, double* grad_table);

#ifdef __cplusplus
}
#endif
#endif
