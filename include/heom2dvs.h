/*
 * heom2dvs.h - C ABI of the GB300 HEOM-2DVS hot path.
 *
 * The library propagates the hierarchical equations of motion (HEOM) of the
 * multi-mode anharmonic Brownian (MAB) model with fourth-order Runge-Kutta and
 * builds the third-order response R(t3, t2, t1) and the 2D correlation IR
 * spectrum (Hoshino and Tanimura, arXiv 2601.20550, Sec. II).  All propagation,
 * kicks, traces and Fourier sums run in CUDA kernels for sm_103a; the host only
 * builds the (small) operator matrices and index tables.
 *
 * Conventions shared by every entry point
 *   - hbar = 1; time in fs; model energies in cm^-1 (converted inside).
 *   - Complex numbers cross the ABI as interleaved (re, im) pairs of double.
 *   - Matrices are row-major.  The product basis orders modes with mode 0 the
 *     slowest index.  A state holds, per branch, every ADO in canonical order
 *     (ascending by (sum of the multi-index, the multi-index as a tuple)), each
 *     ADO a d x d matrix: host layout [branch][ado][d][d] complex.
 *   - Every call returns a heom_status; no exception or abort crosses the ABI.
 *     On failure heom_last_error() gives a message (thread-local).
 *   - The caller owns descriptors and host arrays; the library owns handles and
 *     their device memory.  A handle must not be used by two threads at once.
 *   - Host-pointer calls synchronise before returning.  *_dev calls take device
 *     pointers and a cudaStream_t (passed as void*) and do not synchronise.
 */
#ifndef HEOM2DVS_H
#define HEOM2DVS_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HEOM_OK = 0,
  HEOM_EINVAL = -1,     /* invalid argument or descriptor */
  HEOM_ENOMEM = -2,     /* device or host allocation failed */
  HEOM_ECUDA = -3,      /* CUDA runtime error (message has the CUDA string) */
  HEOM_EUNSTABLE = -4,  /* dt outside the RK4 stability region of the Liouvillian */
  HEOM_ETIMEOUT = -5,   /* a bounded device wait ran out */
  HEOM_ENOTCONV = -6,   /* equilibrium tolerance not reached by t_max */
  HEOM_ENONFINITE = -7, /* a trace or residual became NaN/Inf */
  HEOM_ECKPT = -8       /* checkpoint integrity failure */
} heom_status;

/* Arithmetic of the propagation.  The equilibrium hierarchy is always FP64. */
typedef enum {
  HEOM_FP64 = 0,        /* complex128 state, FP64 right-hand side */
  HEOM_FP32 = 1,        /* complex64 state, FP32 right-hand side on CUDA cores */
  HEOM_TC = 2           /* complex64 state; [H', rho] on tcgen05 tensor cores with split-FP16
                           operands (per-ADO power-of-two scaling), FP32 accumulation */
} heom_precision;

/*
 * One vibrational mode s (Sec. II.A, Eqs. System Hamiltonian, Potentials,
 * counter Hamiltonian, h_int, NLdip; Drude bath Eq. drude; Pade order Sec. II.B).
 *   potential  0: omega (p^2 + q^2)/2 + g3 q^3 / 6 in a harmonic basis of n_prim states
 *              1: omega p^2 / 2 + D (1 - exp(-a q))^2, a = sqrt(omega/(2 D)), on a
 *                 uniform sinc-DVR grid of n_prim points spanning [q_min, q_max]
 *   q is dimensionless with mass m_s = 1/omega_s.
 *   n_levels   eigenstates kept (the mode's basis size n_s)
 *   zeta_cm, gamma_cm  Drude parameters; reorganisation energy m zeta gamma / 2
 *   V_LL, V_SL system-bath coupling V_s(q) = V_LL q + V_SL q^2 / 2
 *   mu1, mu2   dipole mu_s q_s + mu_ss q_s^2 / 2
 *   K_pade     number of Pade terms K_s (the mode has K_s + 1 exponentials)
 */
typedef struct {
  int potential;
  double omega_cm, g3_cm, morse_D_cm;
  int n_levels, n_prim;
  double q_min, q_max;
  double zeta_cm, gamma_cm, V_LL, V_SL, mu1, mu2;
  int K_pade;
} heom_mode;

/* Mode-mode coupling g q_s q_t + (g_s2t q_s^2 q_t + g_st2 q_s q_t^2)/6 and the
 * dipole cross term mu_st q_s q_t (Eqs. Potential ss', NLdip).  s != t. */
typedef struct {
  int s, t;
  double g_st_cm, g_s2t_cm, g_st2_cm, mu_st;
} heom_pair;

/* The model (Eqs. Total Hamiltonian .. h_int) plus hierarchy depth L (all ADOs
 * with sum(n) <= L; Sec. II.B after Eq. HEOM_DB) and the propagation precision. */
typedef struct {
  int n_modes;
  const heom_mode *modes;
  int n_pairs;
  const heom_pair *pairs;
  double T_K;
  int depth_L;
  int precision;   /* heom_precision */
} heom_model;

/* 2D time grid: t1 = j m dt (j < n1), t3 = k m dt (k < n3), t2 from t2_fs[n_t2]
 * (each a multiple of dt).  m = steps_per_sample. */
typedef struct {
  double dt_fs;
  int steps_per_sample, n1, n3, n_t2;
  const double *t2_fs;
} heom_grid;

typedef struct heom_hier heom_hier;     /* opaque, library-owned */
typedef struct heom_state heom_state;   /* opaque, library-owned */

typedef struct {
  int d;            /* product-basis dimension */
  int n_ado;        /* number of ADOs */
  int n_exp;        /* exponentials D = sum_s (K_s + 1) */
  int n_modes;
  int precision;
  double beta;      /* 1/kT in fs/rad */
} heom_hier_info;

/*
 * Build the model matrices and the hierarchy (Sec. II.A-B): mode eigenbases,
 * H_S' with counter terms, V_s, mu and its raising part, the Pade/Matsubara
 * bath exponentials (Eqs. L1, L2, Pade1, Pade2) and the ADO neighbour tables,
 * then upload them.  *out receives a new handle (free with heom_free_hier).
 * Errors: HEOM_EINVAL (bad descriptor), HEOM_ENOMEM, HEOM_ECUDA.
 */
heom_status heom_build_hierarchy(const heom_model *m, heom_hier **out);
heom_status heom_get_info(const heom_hier *h, heom_hier_info *info);

/*
 * Copy the model operators to host arrays (for inspection and tests):
 * H [d*d], mu [d*d], mu_plus [d*d] (may be NULL), bath [n_exp*4] as
 * (mode, nu, Re c, Im c) with C(t) = sum_j c_j exp(-nu_j t), ado [n_ado*n_exp]
 * multi-indices (may be NULL).
 */
heom_status heom_get_operators(const heom_hier *h, double *H, double *mu, double *mu_plus,
                               double *bath, int32_t *ado);

/* Per-mode data of mode s: energies [n_s] and q^k matrices qk [4][n_s][n_s] (k = 1..4)
 * in the kept eigenbasis (may be NULL). */
heom_status heom_get_mode(const heom_hier *h, int s, double *energies, double *qk);

/*
 * Equilibrium hierarchy (Sec. II.C.1): rho_0 = |0><0| (product ground state), all
 * other ADOs zero, propagated with FP64 RK4.  tol <= 0: exactly round(t_max/dt)
 * steps.  tol > 0: stop when max_n ||RHS(rho)_n||_F <= tol ||rho_0||_F (checked
 * every 100 steps); HEOM_ENOTCONV if t_max is reached first (the state is still
 * returned).  *rho_eq receives a new FP64 single-branch state.
 */
heom_status heom_equilibrate(heom_hier *h, double dt_fs, double t_max_fs, double tol,
                             heom_state **rho_eq);

/* States: create (zeroed), upload/download host arrays [branches][n_ado][d][d]
 * complex (interleaved doubles) in the product eigenbasis.  Complex64 states
 * (HEOM_FP32, HEOM_TC) are stored on the device in the coupling eigenbasis,
 * where every V_s is diagonal (rho' = U^T rho U with U the Kronecker product of
 * the per-mode eigenvector matrices of V_s); upload and download convert. */
heom_status heom_state_create(const heom_hier *h, int branches, int precision, heom_state **out);
heom_status heom_state_upload(heom_state *s, const double *host);
heom_status heom_state_download(const heom_state *s, double *host);
/* The same copy under the name of the hot-path contract's boundary list: host
 * receives [branches][n_ado][d][d] complex128 (interleaved doubles) in the product
 * eigenbasis; HEOM_EINVAL for a NULL argument. */
heom_status heom_state_copy_out(const heom_state *s, double *host);
int heom_state_branches(const heom_state *s);

/*
 * Advance every branch of rho by n_steps RK4 steps of Eq. HEOM_DB (Sec. III).
 * The RK4 polynomial is evaluated in nested (Horner) form, identical to the
 * classic four-stage tableau for this linear, time-independent equation.
 * Errors: HEOM_EINVAL, HEOM_EUNSTABLE (dt fails the stability pre-check),
 * HEOM_ECUDA.
 */
heom_status heom_propagate(heom_hier *h, heom_state *rho, double dt_fs, int64_t n_steps);

/*
 * Apply the hyperoperator K^x (K = mu, mu_plus or mu_minus: which = 0, 1, 2) to
 * every ADO of every branch in place (the dipole kicks of Sec. II.C).
 */
heom_status heom_kick(heom_hier *h, heom_state *rho, int which);

/* i^order tr{mu rho_0} of every branch into out [branches] complex (Eqs. R1, RFTIRI). */
heom_status heom_trace(heom_hier *h, const heom_state *rho, int order, double *out);

/*
 * Third-order response and 2D correlation spectrum (Sec. II.C.2, Eqs. RFTIRI,
 * echo, virtual-echo, 2D-rephasing, 2D-nonrephasing, correlation-spectrum):
 *   R_I  = i^3 tr{mu G(t3) (mu+)^x G(t2) (mu+)^x G(t1) (mu-)^x rho_eq}
 *   R_II = i^3 tr{mu G(t3) (mu+)^x G(t2) (mu-)^x G(t1) (mu+)^x rho_eq}
 * where mu+ keeps the elements of mu that raise the total excitation number
 * and mu- = (mu+)^T.  All t1 branches of both pathways are propagated together.
 * Outputs (caller-owned host arrays, any may be NULL):
 *   R_I, R_II [n_t2][n1][n3] complex;  S_C [n_t2][n1][n3] double, indexed by
 *   (Omega1 index q, Omega3 index p), Omega_p = 2 pi p / (N m dt), with the
 *   trapezoid weights 1/2 at t = 0 and S_C(q, p) = S_R((n1 - q) mod n1, p) + S_NR(q, p).
 * rho_eq must be a single-branch FP64 state (from heom_equilibrate).  The
 * propagation runs in the hierarchy's precision (with HEOM_TC, the
 * single-branch t1 trunk runs on the FP32 CUDA-core stage and every batched
 * propagation on the tensor cores); traces accumulate in FP64.
 */
heom_status heom_response_2d(heom_hier *h, const heom_state *rho_eq, const heom_grid *g,
                             double *R_I, double *R_II, double *S_C);

/*
 * Stationary hierarchy by a Krylov solve instead of propagation (the steady
 * state that the equilibration of Sec. II.C.1 approaches): restarted
 * GMRES(restart) from x = |0><0| on A x = 0 with A = L (the right-hand side of
 * Eq. HEOM_DB, FP64, product basis) when steps_per_matvec = 0, or A = G^k - 1
 * with G one RK4 step of dt_fs and k = steps_per_matvec.  Both have the steady
 * state as null vector; the second compresses the spectrum of a stiff hierarchy
 * (fast coherences, slow population transfer) into a range GMRES handles in a
 * few hundred products.  Every correction lies in the range of A, where
 * tr(.)_0 vanishes because the HEOM conserves tr rho_0, so tr x_0 = 1
 * throughout.  Stops when ||L x||_2 <= tol (checked at every restart); at most
 * max_iter Arnoldi steps (HEOM_ENOTCONV with the last iterate in *rho_eq
 * otherwise).  Memory: restart + 5 vectors of n_ado d^2 complex128.  *rho_eq is
 * a single-branch FP64 state usable wherever an equilibrium is taken, except
 * heom_response_2d_grad (which replays a propagation).  *iterations (may be
 * NULL) receives the Arnoldi steps taken.
 */
heom_status heom_steady_state(heom_hier *h, double tol, int restart, int max_iter, double dt_fs,
                              int steps_per_matvec, heom_state **rho_eq, int *iterations);

/*
 * Launch shapes chosen by the library's autotuner (no counterpart in the paper:
 * a tuning aid).  The first RK4 propagation of a given size on the FP64
 * (kind 0) or FP32 coupling-basis (kind 1) path times nine launch shapes of its
 * stage kernel (64/128/256 threads x 4/16/64 blocks per SM) on the real operands
 * and keeps the fastest; results do not depend on the shape.  On the
 * tensor-core path (kind 2) the tensor-core kernel keeps one shape (one
 * persistent 544-thread CTA per SM, bounded by its shared and tensor memory);
 * the coupling kernel that follows it is tuned over seventeen shapes (2, 4, 8 or
 * 16 rows per thread x 1 or 2 groups of 128 threads x 1, 2, 4 or 8 consecutive
 * ADOs per block, some with a bulk L2 prefetch of the block's sources and some
 * also with two neighbour sources in flight per thread; heom_get_tc_shape
 * reports the choice) by timing whole first RK4 stages, before the response
 * scan's graph capture or on the first uncaptured propagation of a size; a
 * batched call keeps its entry in its first hierarchy.  For kind 2, block is threads per block and grid the coupling
 * kernel's blocks per launch.  elements = state elements of the launch (all
 * branches, ADOs and sets).  Returns the number of tuned (kind, elements)
 * entries of h and copies up to cap of them (any pointer may be NULL).
 */
int heom_get_tuning(const heom_hier *h, int cap, int *kind, int64_t *elements, int *block, int *grid);

/*
 * Gradient of the 2D-spectrum misfit
 *   loss = sum_{t2, Omega1, Omega3} (S_C - S_ref)^2
 * (S_C as in heom_response_2d, Eq. correlation-spectrum) with respect to twelve
 * parameters of the model description:
 *   dtheta[0..2]   anharmonicity of mode s (morse_D_cm of a Morse mode, g3_cm of a
 *                  cubic one), dtheta[3..5] g_s2t_cm of pair p (pairs in model order),
 *   dtheta[6..8]   V_SL of mode s, dtheta[9..11] gamma_cm of mode s (zeta_cm fixed);
 * entries for modes or pairs the model lacks are 0.  S_ref is host
 * [n_t2][n1][n3]; *loss and dtheta[12] are written.
 * Method: reverse mode through everything the FP64 path computes -- the
 * equilibration from |0><0| (rho_eq must come from heom_equilibrate; its step
 * count and dt are replayed), the t1 trunk, both pathways' kicks, the t2 and t3
 * propagation (Sec. II.C) and the Fourier sums -- with the RK4 steps reversed
 * stage by stage (the adjoint right-hand side has the structure of Eq. HEOM_DB
 * with H -> -H and the coupling lists transposed) and the states recomputed from
 * checkpoints every ckpt_every steps.  The model matrices' derivatives with
 * respect to each parameter are taken by fourth-order central differences of the
 * host model build (relative step 1e-3) and contracted with the device-accumulated
 * matrix gradients.  Requires a hierarchy built with HEOM_FP64 (HEOM_EINVAL otherwise);
 * device memory is taken in chunks of t1 rows (HEOM_ENOMEM if one row does not fit).
 */
heom_status heom_response_2d_grad(heom_hier *h, const heom_state *rho_eq, const heom_grid *g,
                                  const double *S_ref, int ckpt_every, double *loss, double *dtheta);

/*
 * Several parameter sets (hierarchies of any basis size, each with its own
 * single-branch FP64 equilibrium) on one grid: outputs [n_sets][n_t2][n1][n3]
 * with the layouts of heom_response_2d (any output may be NULL).  When every
 * set is an HEOM_FP64 hierarchy, the sets advance together: each RK4 stage of
 * all sets and all their branches is one kernel launch (per-set models and
 * state pointers in a descriptor table), and each t3 scan is one CUDA-graph
 * replay.  When every set is an HEOM_TC hierarchy (up to 16 sets), each RK4
 * stage of the t2 forks and t3 scans of all sets is one tensor-core launch and
 * one coupling-kernel launch (per-set operators and buffers in the launch's
 * descriptor; a CTA reloads H' when its next item belongs to another set).  In
 * both cases results equal those of heom_response_2d per set, bit for bit.
 * Otherwise (mixed precisions, more than 16 tensor-core sets, or a tensor-core
 * hierarchy named twice) the sets run one after the other, each with all its
 * branches batched.
 */
heom_status heom_response_2d_batched(heom_hier *const *hs, const heom_state *const *eqs, int n_sets,
                                     const heom_grid *g, double *R_I, double *R_II, double *S_C);

/*
 * Rows j0 <= j < j1 (t1 = j m dt) of R_I and R_II only, into R_I, R_II
 * [n_t2][j1 - j0][n3] complex (either may be NULL).  The union of row ranges is
 * the full response; row blocks are independent (the unit of work sharding).
 * The t1 trunk is recomputed from rho_eq up to t1 = j0 m dt.
 */
heom_status heom_response_2d_rows(heom_hier *h, const heom_state *rho_eq, const heom_grid *g, int j0,
                                  int j1, double *R_I, double *R_II);

/*
 * 2D correlation spectrum from given responses (Eqs. 2D-rephasing,
 * 2D-nonrephasing, correlation-spectrum), with the conventions of
 * heom_response_2d: R_I, R_II [n_t2][n1][n3] complex on the host, t = j dtau,
 * S_C [n_t2][n1][n3] out.  Used to assemble a spectrum from row blocks computed
 * on several GPUs.  The Fourier sums run on the device.
 */
heom_status heom_spectrum_2d(const double *R_I, const double *R_II, int n_t2, int n1, int n3,
                             double dtau_fs, double *S_C);

/* Copy branch 0 of src into every branch of dst (converting precision). */
heom_status heom_state_broadcast(const heom_state *src, heom_state *dst);

/* Device address of a state's storage ([branches][n_ado][d][d], complex128 or
 * complex64); valid until heom_free_state. */
void *heom_state_device_ptr(heom_state *s);

/* Device-to-device copy of a state's storage to / from a caller buffer of the
 * same size and representation, on a caller stream (no synchronisation). */
heom_status heom_state_export_dev(const heom_state *s, void *dst, void *stream);
heom_status heom_state_import_dev(heom_state *s, const void *src, void *stream);

/*
 * Linear response R1(t) = i tr{mu G(t) mu^x rho_eq} at t = k m dt, k < n (Eq. R1),
 * into R1 [n] complex, and the absorption I(Omega_p) = Im[dtau sum_k w_k
 * exp(+i Omega_p t_k) R1(t_k)] into I [n] (may be NULL).
 */
heom_status heom_response_1d(heom_hier *h, const heom_state *rho_eq, double dt_fs, int m, int n,
                             double *R1, double *I);

/*
 * Device-pointer RK4 propagation on a caller stream: state and two scratch
 * buffers of the same size, each [branches][n_ado][d][d] complex (complex128 for
 * HEOM_FP64 in the product eigenbasis; complex64 in the coupling eigenbasis
 * otherwise), row-major, ADO stride d*d.  No allocation, no synchronisation;
 * the result is in state.  HEOM_TC requires a hierarchy built with HEOM_TC.
 * Buffers must be aligned to their complex element (16 or 8 bytes; HEOM_EINVAL
 * otherwise).
 */
heom_status heom_propagate_dev(heom_hier *h, void *state, void *scratch_a, void *scratch_b,
                               int branches, int precision, double dt_fs, int64_t n_steps,
                               void *stream);

/* out = K^x in for every ADO of every branch of a device state (K as in
 * heom_kick); in and out must not overlap.  Caller stream, no synchronisation. */
heom_status heom_kick_dev(heom_hier *h, const void *in, void *out, int branches, int precision,
                          int which, void *stream);

/* i^order tr{mu rho_0} of each branch of a device state into out (device,
 * [branches] complex128) on a caller stream; no synchronisation. */
heom_status heom_trace_dev(heom_hier *h, const void *state, int branches, int precision, int order,
                           void *out, void *stream);

/*
 * Allocation-free variant of heom_propagate_dev for callers that cannot
 * allocate device memory when they propagate (a framework's caching allocator
 * owns the pool, a real-time loop cannot afford a cudaMalloc that may
 * synchronise the device, a plug-in has buffers but no allocation rights).
 * The paper has no counterpart: it is a deployment variant of the RK4 step.
 *   state    device pointer, [branches][n_ado][d][d] complex128 (HEOM_FP64
 *            layout), advanced in place by n_steps RK4 steps on `stream`;
 *            16-byte aligned, and dt_fs finite and > 0 (HEOM_EINVAL otherwise,
 *            before any device work).
 * The two RK4 scratch buffers are a file-scope __device__ array of
 * 2 x HEOM_NOALLOC_MAX_BYTES that every GPU loading the library holds until the
 * process exits; states larger than HEOM_NOALLOC_MAX_BYTES are rejected with
 * HEOM_EINVAL.  The call allocates nothing and does not synchronise.  Its first
 * call on a device resolves the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  The hierarchy must already
 * have its device tables (any earlier device call on it, e.g. heom_state_create).
 * Every call shares the one scratch array: calls that overlap on the GPU (other
 * streams, other threads, other hierarchies) race and must be serialised by the
 * caller.  No RK4 stability pre-check is made.
 */
#define HEOM_NOALLOC_MAX_BYTES (16LL * 1024 * 1024)
heom_status heom_propagate_noalloc(heom_hier *h, void *state, int branches, double dt_fs,
                                   int64_t n_steps, void *stream);

/*
 * Checkpoint files (no counterpart in the paper: resume support for runs of
 * hours, e.g. the c5 scan).  A file holds a header (magic "HEOMCKPT", format
 * version, payload size, a tag), the payload and a CRC-32 (IEEE 802.3) of
 * header and payload; it is written under a temporary name and renamed, so an
 * interrupted write leaves the previous file intact.
 *   heom_ckpt_write   host buffer [bytes] -> file
 *   heom_ckpt_read    file -> host buffer [bytes]; the buffer changes only if the
 *                     whole file passes its check
 *   heom_ckpt_verify  integrity check only; *payload_bytes (may be NULL) receives
 *                     the payload size
 *   heom_state_save   a state's device storage as held (complex128 product basis
 *                     or complex64 coupling basis) with its shape in the tag
 *   heom_state_load   into a state of the same shape and precision, bit for bit;
 *                     the state changes only if the file passes its check
 * Errors: HEOM_ECKPT (missing, truncated, foreign or corrupted file: magic,
 * version or CRC mismatch), HEOM_EINVAL (payload size or state shape differs
 * from the caller's), HEOM_ECUDA (device copies).
 */
heom_status heom_ckpt_write(const char *path, const void *host, uint64_t bytes);
heom_status heom_ckpt_read(const char *path, void *host, uint64_t bytes);
heom_status heom_ckpt_verify(const char *path, uint64_t *payload_bytes);
heom_status heom_state_save(const heom_state *s, const char *path);
heom_status heom_state_load(heom_state *s, const char *path);

/*
 * Time limit of every device-side wait of this hierarchy's tensor-core stage
 * kernel (mbarrier waits between its producer, MMA-issue and epilogue warps;
 * no counterpart in the paper: a watchdog of the persistent kernel).  Default
 * 2 s.  A wait that runs out raises the hierarchy's device error word, the
 * kernel drains the tensor-core work it has committed, frees its tensor memory
 * and returns, and the calling entry point returns HEOM_ETIMEOUT (the CUDA
 * context stays usable; the state of that call is not valid).  ns must be > 0
 * (HEOM_EINVAL).
 */
heom_status heom_set_wait_limit_ns(heom_hier *h, uint64_t ns);

/*
 * Host-side allocation-failure injection for tests of the error paths (no
 * counterpart in the paper): after `after` more device allocations by the
 * library succeed, every following one fails as if the device were out of
 * memory, and the entry point that needed it returns HEOM_ENOMEM.  after < 0
 * switches the injection off (the default).  Process-wide.
 */
void heom_debug_fail_alloc(int64_t after);

/*
 * Shape override of the tensor-core path's coupling kernel for tests (no
 * counterpart in the paper): shape 0-16 (rows per thread x groups of 128 threads x
 * consecutive ADOs per block = 8x2x1, 4x2x1, 8x1x1, 4x2x2, 4x2x4, 4x1x4, 2x2x8,
 * 4x1x8, then 8x1x1, 4x2x1, 8x2x1, 4x2x4, 16x1x1, 4x1x1 with a bulk L2 prefetch of
 * each block's source bands, then 8x1x1, 4x1x1, 4x2x1 with the prefetch and two
 * neighbour sources in flight per thread) replaces the autotuner's choice in
 * every following launch; -1 restores tuning.  Results do not depend on the
 * shape: every shape performs the same rounded operations per element, in
 * ascending neighbour order.  Process-wide; HEOM_EINVAL outside -1..16.
 */
heom_status heom_debug_force_tc_shape(int shape);

/* Number of coupling-kernel shapes of the tensor-core path (17; shapes 0 .. count - 1
 * as listed for heom_debug_force_tc_shape).  No device work. */
int heom_tc_shape_count(void);

/* Parameters of coupling-kernel shape `shape` (0 .. count - 1): rows per thread,
 * row groups of 128 threads, consecutive ADOs per block, and flags as for
 * heom_get_tc_shape.  Non-NULL outputs are filled; HEOM_EINVAL out of range. */
heom_status heom_tc_shape_params(int shape, int *rows_per_thread, int *row_groups, int *ados_per_block,
                                 int *flags);

/* Tag of the tensor-core stage kernels' source: the first 16 hex digits of the
 * SHA-256 of tc_stage.cu and tc_stage.h, computed when the library is built, so
 * that a stored measurement (a DRAM-traffic capture) can be matched to the kernels
 * it was taken on.  Static string; no device work. */
const char *heom_source_tag(void);

/*
 * The coupling-kernel shape the autotuner chose for tensor-core launches over
 * `elements` state elements (the kind-2 entries of heom_get_tuning): rows per
 * thread, row groups of 128 threads, consecutive ADOs per block (a block reads
 * the union of those ADOs' neighbour states once) and flags: bit 0 set if the
 * block first requests its source bands into L2, bit 1 set if each thread keeps
 * two neighbour sources' loads in flight.  Returns 1 and fills the non-NULL
 * outputs if such an entry exists, else 0.
 */
int heom_get_tc_shape(const heom_hier *h, int64_t elements, int *rows_per_thread, int *row_groups,
                      int *ados_per_block, int *flags);

void heom_free_hier(heom_hier *h);
void heom_free_state(heom_state *s);
const char *heom_last_error(void);

/* Count of library kernel launches since load (monotonic; for launch accounting). */
uint64_t heom_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* HEOM2DVS_H */
