/*
 * ricmrcc.h -- C ABI of the GB300 spin-free RIC-MRCCSD residual library.
 *
 * The library evaluates the spin-free many-body residual and energy of the
 * renormalized internally contracted multireference coupled cluster method
 * with singles and doubles (RIC-MRCCSD; arXiv 2511.03567, Sec. 2.2-2.3) and
 * solves the amplitude equations with the flow-renormalized update
 * (Eq. ric-update) on one NVIDIA GB300 (sm_103a).
 *
 * Conventions used by every call
 * ------------------------------
 *  - Orbitals are ordered [core | active | virtual]: n = n_core + n_act + n_virt
 *    (Table 1: internal i,j; active t,u,v,...; virtual a,b).
 *  - All floating point data are IEEE double, C (row-major) order.
 *  - Spin-free RDMs use the E-operator convention of Sec. 2.3.1
 *    (Eq. spinfree-spinsum): G1[P*a+Q] = <E^P_Q>, G2[P,Q,R,S] = <E^{PQ}_{RS}>,
 *    G3[P,Q,R,S,T,U] = <E^{PQR}_{STU}>, E^{PQ}_{RS} = sum a+_P a+_Q a_S a_R.
 *  - Spin-free amplitudes are the non-redundant components of Table 2:
 *    singles are the alpha component t^{c}_{k}, doubles the alpha-beta
 *    component t^{c d-bar}_{k l-bar}.  They are passed as one flat array per
 *    rank, the class blocks concatenated in the order reported by
 *    ricmrcc_amplitude_layout():
 *      T1: IA[o][v], IT[o][a], TA[a][v]                (element [k][c] = t^c_k)
 *      T2: IJAB[o][o][v][v], IJTA[o][o][a][v], IJTU[o][o][a][a],
 *          ITAB[o][a][v][v], ITUA[o][a][a][v], ITAU[o][a][v][a],
 *          ITUV[o][a][a][a], TUAB[a][a][v][v], TUVA[a][a][a][v]
 *                                                    (element [k][l][c][d] = t^{cd}_{kl})
 *    ITUA and ITAU are the two stored components of the ITUA class
 *    (Sec. 3.2): t^{u a-bar}_{i t-bar} and t^{a u-bar}_{i t-bar}.
 *    IJAB, IJTU and TUAB must obey t^{cd}_{kl} = t^{dc}_{lk}
 *    (Eq. spinfree-perm-sym); the residual of these classes obeys it too.
 *  - Host pointers are borrowed for the duration of the call and copied;
 *    the handle owns all device memory.  Output buffers are caller-owned.
 *  - *_dev variants take device pointers and run on the handle's stream
 *    (ricmrcc_set_stream); they return after the work is enqueued unless
 *    stated otherwise.
 *  - Every call returns a status code; on failure ricmrcc_last_error()
 *    gives a message owned by the handle (valid until the next call).
 *    No call aborts the process or traps the GPU.
 */
#ifndef RICMRCC_H
#define RICMRCC_H

#include <stdint.h>

#if defined(__GNUC__)
#define RICMRCC_API __attribute__((visibility("default")))
#else
#define RICMRCC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
  RICMRCC_OK = 0,
  RICMRCC_EINVAL = 1,        /* bad argument (size, null pointer, non-finite input) */
  RICMRCC_ENOMEM = 2,        /* device allocation failed */
  RICMRCC_ECUDA = 3,         /* CUDA runtime error */
  RICMRCC_NOT_CONVERGED = 4, /* solve hit max_iter */
  RICMRCC_DIVERGED = 5,      /* non-finite residual/energy or runaway update */
  RICMRCC_ESTATE = 6,        /* call out of order (e.g. residual before set_rdms) */
  RICMRCC_ENOTSUP = 7        /* valid request that this build does not support */
};

/* kind argument of ricmrcc_set_rdms */
enum { RICMRCC_RDM = 0, RICMRCC_CUMULANT = 1 };

/* precision of the dense contractions (ricmrcc_set_precision) */
enum {
  RICMRCC_FP64 = 0,    /* every contraction in FP64 */
  RICMRCC_MIXED = 1,   /* large contractions on BF16 tensor cores (split-precision
                          products, FP32 accumulation), FP64 everything else */
  RICMRCC_EMULATED = 2 /* FP64 accuracy with the large contractions on the BF16
                          tensor cores: the digit-slicing scheme of
                          ricmrcc_gemm_f64_emulated (11 digits), FP64 everything
                          else.  As a solver precision: RICMRCC_MIXED iterations
                          until refine_tol, then iterations at this arithmetic */
};

typedef struct ricmrcc ricmrcc_t;

#define RICMRCC_NCLASS1 3
#define RICMRCC_NCLASS2 9

typedef struct {
  int64_t t1_size;                     /* elements of the flat T1 / R1 array */
  int64_t t2_size;                     /* elements of the flat T2 / R2 array */
  int64_t t1_offset[RICMRCC_NCLASS1];  /* IA, IT, TA */
  int32_t t1_shape[RICMRCC_NCLASS1][2];
  int64_t t2_offset[RICMRCC_NCLASS2];  /* IJAB..TUVA as listed above */
  int32_t t2_shape[RICMRCC_NCLASS2][4];
} ricmrcc_layout;

typedef struct {
  double s;          /* flow parameter s [Eh^-2] of Eq. ric-update; s >= 0 */
  int max_iter;      /* iteration limit (default 100) */
  double e_tol;      /* |E_n - E_{n-1}| threshold (default 1e-10) */
  double t_tol;      /* max |t_new - t| threshold (default 1e-9) */
  int diis_size;     /* DIIS subspace size, 0 disables (default 8) */
  int diis_start;    /* first iteration that extrapolates (default 3) */
  int precision;     /* RICMRCC_FP64, RICMRCC_MIXED or RICMRCC_EMULATED (default FP64) */
  double refine_tol; /* mixed / emulated: switch to FP64-accurate iterations (FP64,
                        resp. emulated FP64) once max|dt| < refine_tol */
} ricmrcc_opts;

typedef struct {
  int iterations;     /* residual evaluations performed */
  int converged;      /* 1 if both thresholds were met */
  int fp64_iterations;
  int mixed_iterations;
  int diverged;       /* 1 if the iteration produced non-finite numbers */
  double energy;      /* E = E0 + Hbar_0 at the returned amplitudes */
  double e0;          /* reference energy <Psi0|H|Psi0> */
  double max_dt;      /* last max |t_new - t| */
  double seconds;     /* wall time of the solve */
} ricmrcc_stats;

/* Create a handle for one problem size (Table 1 spaces) and an auxiliary
 * basis of n_aux functions.  n_core, n_act, n_virt >= 0, n_aux >= 1.
 * n_act = 0 is a single-determinant reference.  Uses the current CUDA device.
 * The many-body residual is RIC-MRCCSD's (RICMRCC_METHOD_RIC).
 * Errors: EINVAL (negative sizes), ENOMEM, ECUDA. */
RICMRCC_API int ricmrcc_create(int n_core, int n_act, int n_virt, int n_aux, ricmrcc_t** out);

/* method argument of ricmrcc_create_method */
enum {
  RICMRCC_METHOD_RIC = 0,  /* H + [H,T] + 1/2[[H,T],T] under the RIC neglect rules (Sec. 2.2) */
  RICMRCC_METHOD_FULL = 1  /* the same expansion without them (cumulants up to lambda_3): the
                              reference point of the neglect error; its term list is ~40 times
                              longer (73 902 residual terms), meant for small systems */
};
/* ricmrcc_create with the residual of `method`.  Every call applies to both
 * methods except ricmrcc_energy_backward (RIC only: ENOTSUP).  Errors as
 * ricmrcc_create, EINVAL for an unknown method. */
RICMRCC_API int ricmrcc_create_method(int n_core, int n_act, int n_virt, int n_aux, int method,
                                      ricmrcc_t** out);

/* Release every resource of the handle (NULL is ignored). */
RICMRCC_API void ricmrcc_destroy(ricmrcc_t* h);

/* Last error message of the handle ("" if none).  Owned by the handle. */
RICMRCC_API const char* ricmrcc_last_error(const ricmrcc_t* h);

/* Stream (cudaStream_t) used by every later call; NULL = legacy default. */
RICMRCC_API int ricmrcc_set_stream(ricmrcc_t* h, void* stream);

/* Select the arithmetic of the dense contractions of ricmrcc_residual and of
 * ricmrcc_step when its options say RICMRCC_FP64 (RICMRCC_FP64 / MIXED /
 * EMULATED). */
RICMRCC_API int ricmrcc_set_precision(ricmrcc_t* h, int precision);

/* One-electron integrals h[n][n] (symmetric) and the density-fitting factor
 * B[n_aux][n][n] (symmetric in the orbital pair), so that the chemist-notation
 * two-electron integral is (pq|rs) = sum_Q B[Q][p][q] B[Q][r][s] and the
 * physicist <pq|rs> = (pr|qs) (Sec. 2.1).  Host pointers.  Rebuilds the
 * integral tensor; if RDMs are already set, also the generalized Fock matrix
 * f = h + sum_C v + sum_A v gamma and E0 (Sec. 2.1).  Errors: EINVAL (NULL
 * or non-finite data). */
RICMRCC_API int ricmrcc_set_integrals(ricmrcc_t* h, const double* hmat, const double* B);
RICMRCC_API int ricmrcc_set_integrals_dev(ricmrcc_t* h, const double* hmat, const double* B);

/* Spin-free reference densities of the CAS state (Sec. 2.3.2, Eq.
 * spinfree-rdm).  kind = RICMRCC_RDM: g1 = Gamma1[a][a], g2 = Gamma2[a]^4,
 * g3 = Gamma3[a]^6.  kind = RICMRCC_CUMULANT: g1 = Gamma1, g2 = Lambda2,
 * g3 = Lambda3 (spin traces of the spin-orbital cumulants of Eq. cumulant and
 * its three-body analogue).  Builds the cumulants used by the residual and,
 * if integrals are set, f and E0.  With n_act = 0 the pointers may be NULL.
 * Host pointers.  Errors: EINVAL. */
RICMRCC_API int ricmrcc_set_rdms(ricmrcc_t* h, const double* g1, const double* g2, const double* g3,
                     int kind);
RICMRCC_API int ricmrcc_set_rdms_dev(ricmrcc_t* h, const double* g1, const double* g2, const double* g3,
                         int kind);

/* Rotate to semi-canonical orbitals (Sec. 2.2: f diagonal inside the core,
 * active and virtual blocks).  Eigenvalues ascend inside each block; each
 * eigenvector's largest-magnitude component is made positive.  Rotates h, B,
 * the RDMs and any stored amplitudes' reference, and rebuilds f, E0.
 * U_out (nullable, host [n][n]) receives new_orbital_j = sum_p U[p][j] old_p.
 * Requires integrals and RDMs.  Errors: ESTATE. */
RICMRCC_API int ricmrcc_semicanonicalize(ricmrcc_t* h, double* U_out);

/* Sizes and offsets of the flat amplitude arrays (see the conventions). */
RICMRCC_API int ricmrcc_amplitude_layout(const ricmrcc_t* h, ricmrcc_layout* out);

/* Reference energy E0 = <Psi0|H|Psi0> (no nuclear repulsion) and the
 * spin-free generalized Fock matrix F[n][n] (alpha component), host outputs;
 * either pointer may be NULL.  Requires integrals and RDMs. */
RICMRCC_API int ricmrcc_reference(ricmrcc_t* h, double* E0, double* F);

/* Many-body residual and energy (Sec. 2.2, Eqs. for E_CC, r^c_k, r^{cd}_{kl}
 * with H-bar truncated after the two-fold commutator and the RIC neglect
 * rules): R = non-redundant spin-free components of H-bar^c_k, H-bar^{cd}_{kl}
 * after Eq. antisym, E = E0 + H-bar_0.  T1/T2 in, R1/R2 out in the flat class
 * layout; E_out (nullable) receives the energy.  Host pointers; blocks until
 * done.  Requires integrals and RDMs.  Errors: ESTATE, EINVAL, ECUDA. */
RICMRCC_API int ricmrcc_residual(ricmrcc_t* h, const double* T1, const double* T2, double* R1, double* R2,
                     double* E_out);
/* Same with device pointers (E_out is a device double, nullable). */
RICMRCC_API int ricmrcc_residual_dev(ricmrcc_t* h, const double* T1, const double* T2, double* R1,
                         double* R2, double* E_out);

/* Fill opts with the defaults listed in ricmrcc_opts. */
RICMRCC_API int ricmrcc_opts_default(ricmrcc_opts* opts);

/* Solve the amplitude equations at flow s [Eh^-2] (s >= 0; it replaces
 * opts->s) with the renormalized update of Eq. ric-update,
 * t <- (t Delta + r)(1 - exp(-s Delta^2)) / Delta with
 * Delta = sum eps(holes) - sum eps(particles), eps = diag f (Eq. cc-update),
 * DIIS-accelerated (Sec. 2.2).  Starts from the stored amplitudes (zero after
 * set_rdms, or those given by ricmrcc_set_amplitudes).  opts (nullable:
 * defaults) sets the thresholds, DIIS and precision.  E_out (nullable) and
 * stats (nullable) receive the result.  Returns OK, NOT_CONVERGED (max_iter
 * reached; amplitudes and energy of the last iterate are kept), DIVERGED
 * (non-finite energy or amplitude change; the amplitudes are left as they
 * were when it was detected) or EINVAL (bad s or options). */
RICMRCC_API int ricmrcc_solve(ricmrcc_t* h, double s, const ricmrcc_opts* opts, double* E_out,
                              ricmrcc_stats* stats);

/* Run n_steps iterations of the solver loop of ricmrcc_solve (residual and
 * energy, Eq. ric-update, DIIS) at flow opts->s without the convergence test,
 * continuing from the stored amplitudes and the DIIS history of earlier
 * calls.  restart != 0 first returns to the solver's initial guess: T = 0
 * and an empty DIIS history.  E_out / max_dt_out (nullable, host) receive
 * the energy at the last evaluated amplitudes and the last max |t_new - t|.
 * Every step uses opts->precision's arithmetic (RICMRCC_EMULATED: emulated
 * FP64 throughout), or the handle's (ricmrcc_set_precision) when that is
 * RICMRCC_FP64.  Returns OK or DIVERGED. */
RICMRCC_API int ricmrcc_step(ricmrcc_t* h, const ricmrcc_opts* opts, int n_steps, int restart,
                             double* E_out, double* max_dt_out);

typedef struct {
  int64_t residual_terms;    /* spin-free terms planned (residual + energy) */
  int64_t residual_launches; /* contraction kernel launches per residual */
  int64_t step_launches;     /* kernel launches per ricmrcc_step iteration */
  double residual_flops;     /* algorithmic FLOPs of one residual + energy */
  double arena_bytes;        /* intermediate arena */
  double table_bytes;        /* offset tables */
  int64_t kind_launches[3];  /* per contraction kernel: 0 = 64x64 tile, 1 = 16x16 tile, 2 = dot */
  double kind_flops[3];
  int64_t tc_contractions;   /* contractions the RICMRCC_MIXED path runs on tensor cores */
  double tc_flops;           /* their FP64-equivalent FLOPs (the BF16 GEMM does 3x) */
  double tc_pack_bytes;      /* algorithmic bytes of their operand packing */
  int64_t graph_launches[2]; /* kernel launches of the captured residual graph [FP64, MIXED]
                                (0 until that graph has been captured) */
  /* per kernel of ricmrcc_profile (same order), for the handle's precision and
   * tile rule: contractions and their FLOPs (tensor-core FLOPs FP64-equivalent;
   * [3], the packing, counts the packed operand buffers and their bytes) */
  int64_t kernel_ops[8];
  double kernel_work[8];
  /* algorithmic bytes of the tensor-core GEMMs per residual: every packed
   * operand buffer read once, every output element read and written once in
   * FP64 per launched op (contractions merged into one op count once; known
   * once the tensor-core path is planned) */
  double tc_gemm_bytes;
  /* ops of the grouped tensor-core launches (merged contractions count once)
   * and how many of them merge contractions of different alphas (+-2^e
   * weights applied inside the MMA); 0 until the tensor-core path is planned
   * with grouped launches */
  int64_t tc_grouped_ops;
  int64_t tc_weighted_ops;
  int64_t oz_contractions;   /* contractions the RICMRCC_EMULATED path runs on tensor cores */
  double oz_flops;           /* their FLOPs (FP64-equivalent) */
} ricmrcc_plan_info_t;

/* Sizes of the contraction program planned for this handle. */
RICMRCC_API int ricmrcc_plan_info(const ricmrcc_t* h, ricmrcc_plan_info_t* out);

/* Time the residual program kernel by kernel with CUDA events on the work
 * stream (reps repetitions, after the caller's warm-up): every contraction
 * runs alone through the kernel the captured residual uses for it.  Returns
 * the mean milliseconds per residual in kind_ms[RICMRCC_PROFILE_KINDS]
 * (host), per kernel: [0] 64x64 tile, [1] 16x16 tile, [2] dot reduction,
 * [3] tensor-core operand packing, [4] tcgen05 GEMM, [5] 128x16 tile,
 * [6] 64x32 tile, [7] small-output long-K reduction.  The tiles compute in
 * FP64, or in FP32 with mixed = 1, which also routes the large contractions
 * to the tensor cores ([3], [4]).  mixed = 2: the RICMRCC_EMULATED schedule,
 * FP64 tiles and the emulated-FP64 contractions (packing included) in [4].
 * Diagnostic: the events serialise the launches. */
#define RICMRCC_PROFILE_KINDS 8
RICMRCC_API int ricmrcc_profile(ricmrcc_t* h, int reps, int mixed, double* kind_ms);

/* Split-precision BF16 tensor-core GEMM (the contraction engine of the
 * RICMRCC_MIXED path, offered on its own):
 *   C[m][n] += alpha * sum_k A[m][k] * B[n][k]
 * A [M][lda], B [N][ldb], C [M][ldc]: row-major FP64 device arrays.  Each
 * operand is split into BF16 hi + lo parts; the product keeps hi*hi, hi*lo and
 * lo*hi (about 16 significant bits) with FP32 accumulation on tcgen05 tensor
 * cores.  Allocates its own temporary device memory; synchronises `stream`.
 * Returns EINVAL (bad sizes), ENOMEM, ENOTSUP (no tensor-map support), ECUDA. */
RICMRCC_API int ricmrcc_gemm_bf16x3(const double* A, int64_t lda, const double* B, int64_t ldb,
                                    double* C, int64_t ldc, int64_t M, int64_t N, int64_t K,
                                    double alpha, void* stream);

/* FP64-accurate GEMM emulated on the BF16 tensor cores (the Ozaki scheme of
 * error-free slicing, Ozaki et al. 2012, in the tensor-core form of
 * Mukunoki et al. 2020; the proposed FP64 route of the refinement steps):
 *   C[m][n] += alpha * sum_k A[m][k] * B[n][k]
 * A [M][lda], B [N][ldb], C [M][ldc]: row-major FP64 device arrays (lda,
 * ldb >= K, ldc >= N).  Each row of alpha*A and of B is scaled by a power of
 * two into (-1, 1) and cut into `slices` signed 5-bit digits (0 = the
 * default RICMRCC_EMULATED_DEFAULT_SLICES, 55 bits; 1 .. MAX allowed); the
 * digit products with i + j < slices run on tcgen05 tensor cores with exact
 * FP32 sums (pieces of at most 8192 products) and are added into C with FP64
 * reductions.  Error per element: at most 4 (slices + 1) 2^{-5 slices} K
 * max_k |alpha A[m][k]| max_k |B[n][k]| from the dropped digits, plus the
 * rounding of the FP64 additions (as in a plain FP64 GEMM).  Cost: slices (slices + 1) / 2 BF16 products.  The
 * order of the FP64 additions varies between runs.  Allocates its own
 * temporary device memory (about 2 slices (M + N) K bytes); synchronises
 * `stream`.  Returns EINVAL (bad sizes or slices, non-finite alpha, or a
 * non-finite entry in A or B, detected before C is touched), ENOMEM,
 * ENOTSUP (no tensor-map support), ECUDA (launch failure or a timed-out
 * pipeline wait). */
#define RICMRCC_EMULATED_DEFAULT_SLICES 11
#define RICMRCC_EMULATED_MAX_SLICES 12
RICMRCC_API int ricmrcc_gemm_f64_emulated(const double* A, int64_t lda, const double* B, int64_t ldb,
                                          double* C, int64_t ldc, int64_t M, int64_t N, int64_t K,
                                          double alpha, int slices, void* stream);

/* Launch only the `count` largest-FLOP contractions of the residual program
 * (largest first), reading the operands left by the last residual.  For
 * profilers that capture one representative launch; blocks until done. */
RICMRCC_API int ricmrcc_run_largest_ops(ricmrcc_t* h, int count);

/* Hand-written adjoint of the converged solve (Sec. 2.2 fixed point of Eq.
 * ric-update): with G(T) = (T Delta + R(T)) phi - T, phi = (1 - exp(-s Delta^2))
 * / Delta, the multipliers solve Lam = (dU/dT)^T Lam + dE/dT (U = G + T, the
 * transposed fixed-point iteration, DIIS-accelerated), and
 *   dE/dtheta = dE/dtheta|_T + Lam . dG/dtheta
 * through the generalized Fock matrix, E0, the integrals and Delta (eps = diag f,
 * the basis is held fixed: no re-canonicalisation).  Outputs (host, nullable):
 * dE_dh [n][n] and dE_dB [n_aux][n][n] with every entry treated as independent
 * (for the symmetric parameters add the transposed entry), dE_ds scalar.
 * Requires the last ricmrcc_solve to have converged (else ESTATE); uses its
 * flow s and options.  The multiplier equations are linear in Lam.  After an
 * FP64 solve they are iterated in FP64.  After a RICMRCC_MIXED solve they
 * are solved by mixed-precision iterative refinement: each outer step takes
 * the FP64 defect r = (dU/dT)^T Lam + dE/dT - Lam, solves the correction
 * delta = (dU/dT)^T delta + r to 1e-3 of |r| with tensor-core (split-BF16,
 * FP32-accumulated) applications of the multiplier terms, and adds delta.
 * Both end at the same FP64 test: max |defect| below max(t_tol, 1e-11).
 * If a refinement step fails to halve the defect, plain FP64 iterations
 * finish.  Returns NOT_CONVERGED / DIVERGED for the multipliers, ECUDA for
 * a timed-out tensor-core wait. */
RICMRCC_API int ricmrcc_energy_backward(ricmrcc_t* h, double* dE_dh, double* dE_dB, double* dE_ds);
/* Same with device outputs (dE_ds a device double), written on the handle's
 * stream; the multiplier iteration still synchronises with the host. */
RICMRCC_API int ricmrcc_energy_backward_dev(ricmrcc_t* h, double* dE_dh, double* dE_dB, double* dE_ds);

/* Work of the last energy_backward call: applications of the multiplier map
 * in FP64 (every term; about 1.5 times the FLOPs of one residual) and in
 * mixed precision (the multiplier terms only), and the wall-clock seconds of
 * the multiplier solve. */
typedef struct ricmrcc_adjoint_info {
  int fp64_applications;
  int mixed_applications;
  double seconds;
} ricmrcc_adjoint_info;
RICMRCC_API int ricmrcc_get_adjoint_info(const ricmrcc_t* h, ricmrcc_adjoint_info* out);

/* Copy the stored amplitudes out / in (flat class layout, host pointers);
 * set_amplitudes allows warm starts and resuming an interrupted solve.
 * set_amplitudes rejects non-finite values (EINVAL). */
RICMRCC_API int ricmrcc_get_amplitudes(ricmrcc_t* h, double* T1, double* T2);
RICMRCC_API int ricmrcc_set_amplitudes(ricmrcc_t* h, const double* T1, const double* T2);
/* Same with device pointers (T1-sized and T2-sized device arrays), enqueued
 * on the handle's stream.  The device variant does not inspect the values:
 * a non-finite amplitude makes the next solver iteration return DIVERGED. */
RICMRCC_API int ricmrcc_get_amplitudes_dev(ricmrcc_t* h, double* T1, double* T2);
RICMRCC_API int ricmrcc_set_amplitudes_dev(ricmrcc_t* h, const double* T1, const double* T2);

/* Residual of the last evaluation (ricmrcc_residual, ricmrcc_step,
 * ricmrcc_solve or ricmrcc_batch_residual / _step / _solve on a batch that
 * owns this handle), in the flat class layout (host pointers T1-sized and
 * T2-sized), at the amplitudes it was evaluated for.  R2 is the
 * pair-symmetrised residual of Eq. antisym, as ricmrcc_residual returns it. */
RICMRCC_API int ricmrcc_get_residual(ricmrcc_t* h, double* R1, double* R2);

/* ---- Kernel choice (tiles) and its autotuner -------------------------------
 *
 * The FP64 contractions of a captured residual run as persistent grouped
 * launches of one of five kernels (64x64, 16x16, 128x16 and 64x32 FP64 output
 * tiles, and a dot reduction); in RICMRCC_MIXED the large GEMM-shaped ones run
 * on the tcgen05 tensor cores instead.  A tile rule fixes both choices:
 *   tc_min_flops  smallest contraction (FLOPs) sent to the tensor cores
 *   skinny        nonzero: tall-skinny contractions (N < 32 <= 64 <= M) use the
 *                 128x16 / 64x32 tiles, else the 16x16 tile.
 *   tc_grouped    nonzero: the tensor-core contractions of a dependency level
 *                 run as one persistent grouped launch, else one launch each.
 *   tc_min_n      smallest output width N sent to the tensor cores (values
 *                 <= 1 admit every N); narrower contractions stay on the
 *                 CUDA-core tiles, where a 128-row MMA tile would be mostly
 *                 padding.
 *   oz_max_pad    RICMRCC_EMULATED: of those, the contractions whose 128 x 256
 *                 x 64 tile padding multiplies the work by at most this factor
 *                 run as emulated-FP64 tensor-core products, the others on the
 *                 FP64 tiles (values below 1 select the default, 4).
 * The result does not depend on the rule beyond rounding. */
typedef struct {
  double tc_min_flops;
  int skinny;
  int tc_grouped;
  int tc_min_n;
  double oz_max_pad;
} ricmrcc_tile_rule;

#define RICMRCC_TUNE_MAX 8
typedef struct {
  int n_candidates;                         /* rules timed */
  ricmrcc_tile_rule rule[RICMRCC_TUNE_MAX]; /* the candidates */
  double ms[RICMRCC_TUNE_MAX];              /* mean residual time of each (CUDA events) */
  int chosen;                               /* index of the fastest; now in effect */
} ricmrcc_tuning;

RICMRCC_API int ricmrcc_set_tile_rule(ricmrcc_t* h, const ricmrcc_tile_rule* rule);
RICMRCC_API int ricmrcc_get_tile_rule(const ricmrcc_t* h, ricmrcc_tile_rule* rule);
/* Time the captured residual under each candidate rule for `precision`
 * (reps timed launches after one warm-up each; changes no amplitudes) and
 * keep the fastest.  The residual is timed at the current amplitudes: tune
 * after a few solver steps, since zero amplitudes skip most accumulations.
 * Needs integrals and RDMs.  out: host, nullable. */
RICMRCC_API int ricmrcc_tune(ricmrcc_t* h, int precision, int reps, ricmrcc_tuning* out);

/* ---- Batched instances -----------------------------------------------------
 *
 * Many independent problems of uneven sizes solved together on one GPU.  Each
 * iteration evaluates every instance's residual in one CUDA graph whose
 * dependency levels ("waves") are each one persistent grouped launch per FP64
 * tile kind over the contractions of all instances (plus the instances'
 * tensor-core contractions in RICMRCC_MIXED); the renormalised update and DIIS
 * then run per instance, with one host synchronisation per phase for the
 * whole batch.  Results equal those of solving each instance on its own
 * (ricmrcc_solve) up to the accumulation order of the atomic reductions. */
typedef struct ricmrcc_batch ricmrcc_batch_t;

/* dims[i] = {n_core, n_act, n_virt, n_aux} of instance i (count >= 1).
 * Instances are planned in parallel host threads. */
RICMRCC_API int ricmrcc_batch_create(int count, const int (*dims)[4], ricmrcc_batch_t** out);
RICMRCC_API void ricmrcc_batch_destroy(ricmrcc_batch_t* b);
RICMRCC_API const char* ricmrcc_batch_last_error(const ricmrcc_batch_t* b);
/* Borrowed handle of instance i (owned by the batch: never destroy it).  All
 * single-instance calls apply to it: set_integrals, set_rdms,
 * semicanonicalize, amplitude_layout, get/set_amplitudes, get_residual, ... */
RICMRCC_API int ricmrcc_batch_instance(ricmrcc_batch_t* b, int i, ricmrcc_t** out);
/* Shorthands for ricmrcc_set_integrals / ricmrcc_set_rdms on instance i. */
RICMRCC_API int ricmrcc_batch_set_integrals(ricmrcc_batch_t* b, int i, const double* h, const double* B);
RICMRCC_API int ricmrcc_batch_set_rdms(ricmrcc_batch_t* b, int i, const double* g1, const double* g2,
                                       const double* g3, int kind);
/* Residuals and energies of all instances at their current amplitudes, in
 * `precision` (RICMRCC_FP64 / RICMRCC_MIXED).  E_out: host [count], nullable;
 * read the residuals with ricmrcc_get_residual on the instances. */
RICMRCC_API int ricmrcc_batch_residual(ricmrcc_batch_t* b, int precision, double* E_out);
/* Solve all instances with one set of options (precision, flow s, ...;
 * RICMRCC_FP64 or RICMRCC_MIXED, RICMRCC_EMULATED is refused with EINVAL, as
 * in ricmrcc_batch_step).  In
 * RICMRCC_MIXED every instance iterates on the tensor-core path until all
 * unconverged instances reach max|dt| < refine_tol, then the batch refines in
 * FP64.  Converged instances stop updating; the graph drops them once half of
 * its instances have finished.  E_out: host [count]; stats: host [count],
 * nullable.  Returns OK when all converged, else NOT_CONVERGED or DIVERGED
 * (the per-instance outcome is in stats). */
RICMRCC_API int ricmrcc_batch_solve(ricmrcc_batch_t* b, const ricmrcc_opts* opts, double* E_out,
                                    ricmrcc_stats* stats);
/* ricmrcc_batch_solve with a flow value per instance (s[count], host; it
 * replaces opts->s): a scan of the flow parameter over copies of one problem
 * runs as one batch (the paper's accuracy-vs-s and non-convergence study,
 * Sec. 4).  Per-instance outcomes (converged / diverged, iterations, max|dt|)
 * are in stats; a diverged instance stops updating and does not stop the
 * others. */
RICMRCC_API int ricmrcc_batch_solve_flows(ricmrcc_batch_t* b, const double* s, const ricmrcc_opts* opts,
                                          double* E_out, ricmrcc_stats* stats);
/* n_steps batch iterations without convergence tests (restart != 0 resets the
 * DIIS histories).  E_out, max_dt_out: host [count], nullable. */
RICMRCC_API int ricmrcc_batch_step(ricmrcc_batch_t* b, const ricmrcc_opts* opts, int n_steps, int restart,
                                   double* E_out, double* max_dt_out);
/* ricmrcc_tune for the batch graph: one rule for all instances. */
RICMRCC_API int ricmrcc_batch_tune(ricmrcc_batch_t* b, int precision, int reps, ricmrcc_tuning* out);
/* Sizes of the last captured batch graph: waves (dependency levels), grouped
 * FP64 launches, tensor-core contractions and FP64-equivalent FLOPs per
 * iteration over all instances. */
typedef struct {
  int waves;
  int64_t grouped_launches;
  int64_t tc_contractions;
  double flops;
  double tc_flops;
  int64_t kernel_launches; /* kernel launches of one batch residual graph */
} ricmrcc_batch_info_t;
RICMRCC_API int ricmrcc_batch_info(const ricmrcc_batch_t* b, ricmrcc_batch_info_t* out);

/* ---- Density-fitted particle-particle ladder -------------------------------
 *
 * The linear vvvv term of the doubles residual (Sec. 2.2; the contraction
 * Sec. 4.3 names rate-limiting), with the integrals rebuilt from the
 * density-fitting factor inside the call:
 *   R^{ab}_{kl} += sum_{e,f virtual} (ae|bf) T^{ef}_{kl},  (ae|bf) = sum_Q B[Q][a][e] B[Q][b][f]
 * for all hole pairs (k, l) (core and active: n_hole = n_core + n_act) and
 * virtual a, b.  For systems whose integral tensor does not fit in memory
 * (v^4 numbers): the integrals exist only one slab of pairs (a, b) at a time.
 * Arithmetic: split-precision BF16 products (hi*hi + hi*lo + lo*hi, about 16
 * significant bits per operand) with FP32 accumulation on the tcgen05 tensor
 * cores, both for the integral rebuild and for the ladder; R accumulates in
 * FP64.  The amplitudes must be pair-symmetric, T^{ef}_{kl} = T^{fe}_{lk}
 * (Eq. spinfree-perm-sym); the work uses the (e,f)-symmetric and
 * -antisymmetric parts, a quarter of the unpacked products.
 *
 * Layouts (row-major FP64): Bvv[n_aux][n_virt][n_virt] (the virtual-virtual
 * block of ricmrcc_set_integrals' B, symmetric in the orbital pair);
 * T and R [n_hole][n_hole][n_virt][n_virt], element [k][l][e][f] = T^{ef}_{kl}.
 * The handle owns its device workspace (ricmrcc_ladder_info reports it;
 * ENOMEM at create if it does not fit). */
typedef struct ricmrcc_ladder ricmrcc_ladder_t;
typedef struct {
  int slabs;                      /* slabs of pairs (a, b) per application */
  int64_t slab_rows;              /* largest slab (pairs a <= b) */
  double rebuild_flops;           /* algorithmic: 2 n_aux per integral (ae|bf), a <= b: n_aux v^3 (v+1) */
  double ladder_flops;            /* algorithmic, symmetric/antisymmetric packed products */
  double rebuild_flops_executed;  /* BF16 tensor-core FLOPs issued (3 products, padding) */
  double ladder_flops_executed;
  double workspace_bytes;
  /* milliseconds of the last application, per phase (CUDA events on the
   * handle's stream; filled by ricmrcc_ladder_finish) */
  double ms_pack, ms_rebuild, ms_symmetrise, ms_ladder, ms_unpack;
} ricmrcc_ladder_info_t;

/* n_hole, n_virt, n_aux >= 1; slab_rows = largest number of pairs (a <= b)
 * per slab (0: 12288; a slab also spans at most 24 values of a).  Uses the current CUDA device.  Errors: EINVAL,
 * ENOMEM, ENOTSUP (no tensor-map support), ECUDA. */
RICMRCC_API int ricmrcc_ladder_create(int n_hole, int n_virt, int n_aux, int64_t slab_rows,
                                      ricmrcc_ladder_t** out);
RICMRCC_API void ricmrcc_ladder_destroy(ricmrcc_ladder_t* L);
RICMRCC_API const char* ricmrcc_ladder_last_error(const ricmrcc_ladder_t* L);
/* Stream the calls are ordered after and before (NULL = legacy default). */
RICMRCC_API int ricmrcc_ladder_set_stream(ricmrcc_ladder_t* L, void* stream);
/* Pack the factor (kept until the next call).  Device pointer; enqueued. */
RICMRCC_API int ricmrcc_ladder_set_factor_dev(ricmrcc_ladder_t* L, const double* Bvv);
/* R += ladder(T).  Device pointers; enqueued: ricmrcc_ladder_finish waits
 * for it and reports its status.  Errors: ESTATE (no factor), EINVAL. */
RICMRCC_API int ricmrcc_ladder_apply_dev(ricmrcc_ladder_t* L, const double* T, double* R);
/* Wait for the enqueued work; out (nullable) receives the sizes and the
 * phase times of the last application.  Returns ECUDA if a tensor-core
 * pipeline wait timed out (the kernels stopped; the context stays usable). */
RICMRCC_API int ricmrcc_ladder_finish(ricmrcc_ladder_t* L, ricmrcc_ladder_info_t* out);
/* Sizes and algorithmic work (no waiting). */
RICMRCC_API int ricmrcc_ladder_info(ricmrcc_ladder_t* L, ricmrcc_ladder_info_t* out);
/* Host-pointer variants (copy in and out; blocking). */
RICMRCC_API int ricmrcc_ladder_set_factor(ricmrcc_ladder_t* L, const double* Bvv);
RICMRCC_API int ricmrcc_ladder_apply(ricmrcc_ladder_t* L, const double* T, double* R);

/* Time bound of every wait inside the tensor-core kernels (seconds, > 0;
 * default 4).  A wait that runs out sets the call's error status (ECUDA,
 * "tensor-core pipeline wait timed out"); the kernels stop after their
 * copies and MMAs in flight have landed, so the context stays usable.
 * stall_test != 0 makes every tensor-core kernel launched afterwards first
 * wait on a barrier that nothing completes, so that wait runs out after
 * `seconds`: a test of that error path without any fault (0 for normal
 * work).  Applies to kernels launched afterwards on the current device; call
 * it outside stream capture. */
RICMRCC_API int ricmrcc_set_wait_limit(double seconds, int stall_test);

/* Allocation-free eigensolver for one symmetric block (no counterpart in the
 * paper; it is the eigen-step of ricmrcc_semicanonicalize offered on its own).
 *
 * For callers that cannot allocate device memory when they need it: code
 * running while a stream is captured into a CUDA graph, services that reserve
 * their whole device-memory budget up front, or hosts whose allocator belongs
 * to another runtime.  The call allocates nothing (no cudaMalloc, cudaFree or
 * allocating library routine); its working memory is one fixed device array
 * of 2 * RICMRCC_NOALLOC_MAX_N^2 doubles (16 MiB) inside the library, which
 * every device that loads the library keeps until the process exits.
 *
 * A: device pointer to a symmetric n x n row-major matrix (read only).
 * eigenvalues: device [n], ascending.  eigenvectors: device [n][n], column j
 * belongs to eigenvalue j and its largest-magnitude component is positive
 * (the conventions of ricmrcc_semicanonicalize).  stream: cudaStream_t (NULL
 * = legacy default); the call returns once the work is enqueued.  The
 * eigen-decomposition is a cyclic Jacobi iteration in one thread block
 * (about n^3 work per sweep; measured on a GB300: 1.6 s per call at n = 300,
 * 40 s at n = 1000, milliseconds for the blocks of a few dozen orbitals of
 * the semi-canonicalisation).  If 40 sweeps leave the block unconverged, every eigenvalue is
 * NaN: the call only enqueues work, so the outcome reaches the caller that
 * way.  Returns EINVAL for NULL pointers, n < 1 or n > RICMRCC_NOALLOC_MAX_N,
 * and ECUDA if the device address of the working array cannot be obtained or
 * one of this call's own launches fails.
 *
 * The first call on each device looks up that device's address of the
 * working array (with the device current); make that first call before any
 * stream capture.  All calls share the one working array: calls whose GPU
 * work overlaps (different streams, or different host threads) race and
 * corrupt each other's results; serialise them. */
#define RICMRCC_NOALLOC_MAX_N 1024
RICMRCC_API int ricmrcc_block_eigh_noalloc(const double* A, int n, double* eigenvalues,
                                           double* eigenvectors, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RICMRCC_H */
