/*
 * cheb_expmv.h - C ABI of the B300 (sm_103a) library for psi(t) = exp(-i t H) psi,
 * H = H_P + gamma * sum_j X_j on n qubits, evaluated as a truncated Chebyshev or
 * Caratheodory-Fejer series with the matrix Clenshaw recurrence and a matrix-free
 * hypercube matvec (Hopkins & Kendon, "Numerical methods for the simulation of
 * quantum walks and quantum annealing").
 *
 * Conventions shared by every entry point
 *   - n qubits, N = 2^n basis states; basis index z, qubit i is bit i of z (least
 *     significant first), spin s_i(z) = 1 - 2*bit_i(z).
 *   - Ising diagonal (Sec. I): E(z) = sum_{i<j} J[i*n+j] s_i s_j + sum_i h[i] s_i.
 *     h has n doubles, J is an n x n row-major matrix of doubles of which only the
 *     strict upper triangle (i < j) is read. Both are HOST pointers, read during
 *     the call and not retained.
 *   - States are DEVICE pointers to N interleaved complex numbers: complex64
 *     (float re, float im) for CHEB_FP32, complex128 (double re, double im) for
 *     CHEB_FP64, 16-byte aligned. The caller owns them.
 *   - workspace is a DEVICE buffer of at least cheb_workspace_bytes(...) bytes,
 *     256-byte aligned, owned by the caller; the library allocates no device
 *     memory. Calls that share a workspace must not overlap on the GPU.
 *   - stream is a cudaStream_t (NULL = legacy default stream). Work is enqueued on
 *     it. Entry points that need a device result on the host (the spectral bounds,
 *     or anything written to an info struct) synchronise that stream.
 *   - Errors are returned as cheb_status_t, never by exit or exception. Argument
 *     errors are detected before any work is enqueued. Device-side conditions
 *     (non-finite results, a wait that ran out) are reported when the call
 *     synchronises (i.e. when an info struct is requested).
 */
#ifndef CHEB_EXPMV_H
#define CHEB_EXPMV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CHEB_OK = 0,
    CHEB_ERR_INVALID_ARG = 1,   /* bad size, null pointer, non-finite scalar, bad enum */
    CHEB_ERR_WORKSPACE = 2,     /* workspace too small or misaligned */
    CHEB_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    CHEB_ERR_TIMEOUT = 4,       /* a bounded device-side wait ran out */
    CHEB_ERR_NONFINITE = 5,     /* the result contains NaN or Inf */
    CHEB_ERR_UNSUPPORTED = 6    /* valid but outside what this build handles */
} cheb_status_t;

typedef enum { CHEB_METHOD_CHEBYSHEV = 0, CHEB_METHOD_CF = 1, CHEB_METHOD_REMEZ = 2 } cheb_method_t;
typedef enum { CHEB_FP32 = 0, CHEB_FP64 = 1 } cheb_precision_t;

/* Kernel path for the Clenshaw steps. AUTO picks the fastest path measured for
 * (n, precision): the whole run in one CTA's shared memory for n <= 13 (FP32) or 12
 * (FP64), the plain kernel up to n = 19 (FP32) or 16 (FP64), the fused kernels above;
 * batches run instances of n = 14..17 (FP32) or 13..16 (FP64) on clusters. PLAIN
 * forces the one-pass kernel that reads every bit-flip partner from global memory
 * (the reference GPU path; for FP64 it is the native FP64 recurrence); FUSED forces
 * the shared-memory tiled kernels (n >= 11; for FP64 these keep complex128 storage and
 * compute in float-float on the FP32 units, about 48 significant bits, see
 * cheb_set_fused_split_fp64); CLUSTER forces the whole run on one thread-block cluster
 * with the vectors in distributed shared memory (FP32 n = 14..17, FP64 n = 13..16;
 * UNSUPPORTED elsewhere or if the device has no room for such a cluster). */
typedef enum {
    CHEB_PATH_AUTO = 0,
    CHEB_PATH_PLAIN = 1,
    CHEB_PATH_FUSED = 2,
    CHEB_PATH_CLUSTER = 3
} cheb_path_t;

typedef struct {
    int K;               /* polynomial degree per time slice (matvecs per slice) */
    int time_splits;     /* number of equal time slices */
    int64_t matvecs;     /* total operator applications = K * time_splits */
    double emin, emax;   /* range of the Ising diagonal E(z) */
    double center;       /* c = (emax + emin) / 2, the spectral shift (Sec. II.A) */
    double radius;       /* r = (emax - emin) / 2 + |gamma| n = ||H - c||_1 (Sec. II.A) */
    double a;            /* (t / time_splits) * r, the argument of the series */
    double trunc_bound;  /* truncation bound (Eq. TruncError) or CF estimate, summed over slices */
    double norm;         /* ||y||_2, FP64 reduction on the device */
    double energy;       /* <y|H_P|y>, FP64 reduction on the device */
    double eval_bound;   /* a-posteriori evaluation-error bound of Sec. II.B.3 (absolute, 2-norm,
                            summed over slices) when CHEB_FLAG_EVAL_BOUND was given, else -1 */
} cheb_info_t;

/* Flag OR-ed into the `path` argument of cheb_expmv_path: also compute the evaluation-
 * error bound of Sec. II.B.3 (analysis of evaluation error),
 *   sum_{k=0}^{K} u ||b_k|| + u ||c_k psi - b_{k+2}|| + sqrt(d) gamma_d ||b_{k+1}||,
 * with b_0 = y, d = n + 1 nonzeros per column of H, gamma_d = d u / (1 - d u) and u the
 * unit roundoff of the arithmetic (2^-24 for CHEB_FP32; 2^-47 for the float-float
 * fused FP64 step; 2^-53 for the native FP64 kernels), from FP64 norms of every
 * Clenshaw vector reduced on the device after each step. It needs every b_k in memory,
 * so the whole-run shared-memory kernel is replaced by PLAIN (CLUSTER is UNSUPPORTED);
 * it costs one extra read of b_k and psi per step and synchronises once per time
 * slice. Requires info (INVALID_ARG otherwise). */
#define CHEB_FLAG_EVAL_BOUND 0x100

/* Human-readable name of a status code (static string). */
const char* cheb_status_string(cheb_status_t status);

/* Library version string (static). */
const char* cheb_version(void);

/*
 * Host coefficient generator (Sec. II.B.1, Eq. cheb, Eq. TruncError; Sec. II.C for CF and Remez).
 * Coefficients of f(x) = exp(-i a x) * phase on [-1, 1] in the Chebyshev basis,
 * c_0 = J_0(a) * phase, c_m = 2 (-i)^m J_m(a) * phase (CHEB_METHOD_CHEBYSHEV), the
 * Caratheodory-Fejer near-minimax correction of that series (CHEB_METHOD_CF), or the
 * minimax polynomials of cos(a x) and sin(a x) from the Remez exchange
 * (CHEB_METHOD_REMEZ, Sec. II.C; err_bound = hypot of their minimax errors).
 * K is the smallest degree whose truncation bound sum_{m>K} |c_m| (Chebyshev) or
 * CF error estimate is <= tol.
 *   coeffs:  HOST buffer of 2*(max_K+1) doubles, receives (re, im) of c_0..c_K.
 *   K:       receives the degree. err_bound (nullable) receives the bound/estimate.
 * Errors: INVALID_ARG (non-finite a, tol <= 0, bad method, null pointers),
 *         UNSUPPORTED (K would exceed max_K).
 */
cheb_status_t cheb_coefficients(double a, double phase_re, double phase_im, double tol,
                                cheb_method_t method, int max_K, double* coeffs, int* K,
                                double* err_bound);

/* Workspace bytes needed by cheb_expmv / cheb_ising_bounds / cheb_energy at
 * (n, precision). Returns 0 for an unsupported n (outside 1..33). */
size_t cheb_workspace_bytes(int n, cheb_precision_t precision);

/*
 * Spectral bounds (Sec. II.A): exact minimum and maximum of E(z) over all 2^n basis
 * states, computed on the device from the couplings (energies are summed exactly
 * in 64-bit fixed point). Synchronises the stream.
 *   emin, emax: HOST outputs.
 */
cheb_status_t cheb_ising_bounds(int n, const double* h, const double* J, void* workspace,
                                size_t workspace_bytes, void* stream, double* emin, double* emax);

/*
 * psi <- exp(-i t H) psi, H = diag(E) + gamma * sum_j X_j (Sec. I).
 * Pipeline: spectral bounds c, r (Sec. II.A); for each of the time slices,
 * coefficients of exp(-i a x) with a = (t/s) r and the global phase exp(-i (t/s) c)
 * (Eq. cheb, Eq. TruncError / Sec. II.C); the matrix Clenshaw recurrence
 * (Algorithm 2, Eq. recursion) with Ht = (H - c)/r applied matrix-free (Sec. II.D),
 * b_k written in place over b_{k+2}, the result written into psi.
 *   psi:          DEVICE in/out, N complex numbers of the given precision.
 *   tol:          bound on the truncation error per unit norm, split evenly over slices.
 *   time_splits:  number of slices s >= 1, or 0 for automatic (1 unless the degree
 *                 would exceed the coefficient table, 65536).
 *   info:         nullable; when given, the call synchronises and fills it (including
 *                 the FP64 norm and energy of the result).
 * Errors: INVALID_ARG, WORKSPACE, CUDA, NONFINITE (info given and y not finite),
 *         UNSUPPORTED.
 */
cheb_status_t cheb_expmv(int n, const double* h, const double* J, double gamma, double t,
                         void* psi, cheb_precision_t precision, double tol, cheb_method_t method,
                         int time_splits, void* workspace, size_t workspace_bytes, void* stream,
                         cheb_info_t* info);

/*
 * cheb_expmv_noalloc: cheb_expmv without a caller-supplied workspace. The paper has
 * no counterpart; it exists for callers that cannot allocate device memory (code
 * running inside a pool or allocator that forbids foreign cudaMalloc calls, plugins
 * that only receive their input and output buffers, programs that must not grow
 * their device footprint after start-up).
 *   - Scratch: a fixed 10 MiB array inside the library image (a __device__ array),
 *     held by every GPU that loads the library's device code until the process
 *     exits. It is enough for n <= 19 in FP32 and n <= 18 in FP64; larger n returns
 *     CHEB_ERR_UNSUPPORTED before any work is enqueued.
 *   - The call allocates nothing: no cudaMalloc, cudaFree or allocating library
 *     routine. psi (device, in/out), h, J and info are as for cheb_expmv.
 *   - The first call on each device looks up the array's device address (with that
 *     device current) and caches it; make that first call before any stream capture.
 *     The cache is keyed on the device's context, so after a context reset
 *     (cudaDeviceReset) the next call looks the address up again.
 *   - A device-side condition (a bounded wait that ran out) is only reported through
 *     info: pass info to learn it.
 *   - All calls share the one array. Calls that overlap on the GPU (other streams,
 *     other host threads on the same device) race on it and must be serialised by
 *     the caller.
 * Errors: as cheb_expmv, plus UNSUPPORTED for sizes beyond the scratch array.
 */
cheb_status_t cheb_expmv_noalloc(int n, const double* h, const double* J, double gamma, double t,
                                 void* psi, cheb_precision_t precision, double tol,
                                 cheb_method_t method, int time_splits, void* stream,
                                 cheb_info_t* info);

/*
 * Piecewise-constant annealing schedule (the constant-H building block of the
 * time-dependent evolution of Sec. III.B): for s = 0..S-1,
 *   psi <- exp(-i t_s H_s) psi,   H_s = diag(E) + gamma_s sum_j X_j.
 * The spectral scan runs once (E is shared); each segment uses its own radius
 * r_s = (Emax - Emin)/2 + |gamma_s| n and series (Eq. cheb / Sec. II.C) with
 * tolerance tol / S, so the whole schedule meets tol in the truncation bound.
 *   gamma_s, t_s: HOST arrays of S doubles.
 *   boundaries:   nullable DEVICE buffer of S states (S * 2^n complex of the given
 *                 precision); receives the state at the start of each segment.
 *   infos:        nullable HOST array of S cheb_info_t (per segment; norm and energy
 *                 of the state after that segment). Requesting infos synchronises
 *                 the stream once per segment.
 * Workspace: cheb_workspace_bytes(n, precision). Errors: as cheb_expmv.
 */
cheb_status_t cheb_anneal(int n, const double* h, const double* J, int S, const double* gamma_s,
                          const double* t_s, void* psi, cheb_precision_t precision, double tol,
                          cheb_method_t method, void* boundaries, void* workspace,
                          size_t workspace_bytes, void* stream, cheb_info_t* infos);

/*
 * General piecewise-constant schedule H_s = b_s diag(E) + a_s sum_j X_j (the usual
 * annealing form A(t) H_X + B(t) H_P sampled per segment; cheb_anneal is b_s = 1):
 * psi <- exp(-i t_s H_s) psi for s = 0..S-1. b_s may be zero or negative: b_s H_P
 * has centre b_s c and half-width |b_s| (Emax - Emin)/2, from one spectral scan.
 *   a_s, b_s, t_s: HOST arrays of S doubles. Other arguments as cheb_anneal; the
 *   energy in infos is that of the segment's diagonal part b_s H_P.
 * Errors: as cheb_anneal.
 */
cheb_status_t cheb_anneal_general(int n, const double* h, const double* J, int S, const double* a_s,
                                  const double* b_s, const double* t_s, void* psi,
                                  cheb_precision_t precision, double tol, cheb_method_t method,
                                  void* boundaries, void* workspace, size_t workspace_bytes,
                                  void* stream, cheb_info_t* infos);

/*
 * CUDA-graph capture of a schedule (no counterpart in the paper). cheb_anneal_graph_create
 * runs the host side of cheb_anneal_general once (spectral scan, fixed-point couplings,
 * series and degrees of every segment; it synchronises the stream), keeps each
 * segment's couplings in the workspace, and captures the device work of the whole
 * schedule into a graph: per segment the boundary copy, the table rebuild and the
 * Clenshaw steps, on the same kernels as cheb_anneal_general. cheb_anneal_graph_launch
 * replays it on `stream`: psi <- prod_s exp(-i t_s H_s) psi again, bit for bit what
 * cheb_anneal_general computes from the same state.
 *   Arguments as cheb_anneal_general (b_s null means b_s = 1, i.e. cheb_anneal).
 *   psi, boundaries and workspace are bound into the graph: they must stay allocated
 *   and are the buffers every replay reads and writes.
 *   workspace: cheb_anneal_graph_workspace_bytes(n, precision, S) bytes, 256-byte
 *   aligned, used only by this graph while it exists.
 *   graph: HOST out; release with cheb_anneal_graph_destroy.
 * A replay does not synchronise; its bounded waits report through the workspace's
 * status word (cheb_workspace_status). Replays count their kernels in
 * cheb_launch_count. Errors: as cheb_anneal_general; UNSUPPORTED while per-kernel event
 * timing is on (cheb_profile_enable); CUDA if the capture or instantiation fails.
 */
typedef struct cheb_anneal_graph* cheb_anneal_graph_t;
size_t cheb_anneal_graph_workspace_bytes(int n, cheb_precision_t precision, int S);
cheb_status_t cheb_anneal_graph_create(int n, const double* h, const double* J, int S,
                                       const double* a_s, const double* b_s, const double* t_s,
                                       void* psi, cheb_precision_t precision, double tol,
                                       cheb_method_t method, void* boundaries, void* workspace,
                                       size_t workspace_bytes, void* stream,
                                       cheb_anneal_graph_t* graph);
cheb_status_t cheb_anneal_graph_launch(cheb_anneal_graph_t graph, void* stream);
void cheb_anneal_graph_destroy(cheb_anneal_graph_t graph);

/*
 * Time-dependent evolution i dpsi/dt = H(t) psi with H(t) = A(t) sum_j X_j + B(t) H_P
 * by the fourth-order commutator-free Magnus integrator that Sec. III.B builds on:
 * per step of length dt_m, with Gauss-Legendre nodes t1,2 = t + (1/2 -+ sqrt(3)/6) dt_m,
 *   psi <- exp(-i dt (w1 H(t1) + w2 H(t2))) exp(-i dt (w2 H(t1) + w1 H(t2))) psi,
 *   w1 = 1/4 - sqrt(3)/6, w2 = 1/4 + sqrt(3)/6
 * (the right factor first). Each factor is one segment of cheb_anneal_general.
 *   dt:     HOST array of `steps` step lengths.
 *   nodes:  HOST array of 4*steps doubles: A(t1), B(t1), A(t2), B(t2) per step.
 *   tol:    truncation budget of all 2*steps exponentials together (the integrator's
 *           own O(dt^5) local error is the caller's choice of steps).
 *   boundaries: nullable DEVICE buffer of 2*steps states; receives the state before
 *           each exponential (for cheb_magnus4_adjoint).
 *   infos:  nullable HOST array of 2*steps cheb_info_t (one per exponential).
 * Workspace: cheb_workspace_bytes(n, precision). Errors: INVALID_ARG (steps < 1,
 * null or non-finite dt/nodes), otherwise as cheb_anneal.
 */
cheb_status_t cheb_magnus4(int n, const double* h, const double* J, int steps, const double* dt,
                           const double* nodes, void* psi, cheb_precision_t precision, double tol,
                           cheb_method_t method, void* boundaries, void* workspace, size_t workspace_bytes,
                           void* stream, cheb_info_t* infos);

/* A schedule for the Magnus entry points: writes A(t) and B(t) of
 * H(t) = A(t) sum_j X_j + B(t) H_P; returns 0 on success (anything else aborts the
 * call with CHEB_ERR_INVALID_ARG). Called on the calling host thread. */
typedef int (*cheb_schedule_fn)(double t, double* A, double* B, void* user);

/*
 * Samples a schedule for cheb_magnus4 on `steps` equal steps of [0, T]: dt[m] = T/steps
 * and nodes[4m..4m+3] = A(t1), B(t1), A(t2), B(t2) at the Gauss-Legendre points
 * t1,2 = m dt + (1/2 -+ sqrt(3)/6) dt.
 *   dt, nodes: HOST outputs of steps and 4*steps doubles.
 * Errors: INVALID_ARG (steps < 1, null pointers, non-finite T or schedule values).
 */
cheb_status_t cheb_magnus4_nodes(double T, int steps, cheb_schedule_fn schedule, void* user, double* dt,
                                 double* nodes);

/*
 * Reverse-mode gradients of cheb_magnus4 (no counterpart in the paper): the adjoint of
 * its 2*steps exponentials (cheb_anneal_general_adjoint) chained through the
 * Gauss-node combinations, so that gradients reach every step length and node value:
 *   dL/d dt_m = dL/dt_{2m} + dL/dt_{2m+1},
 *   dL/dA(t1) = w2 dL/da_{2m} + w1 dL/da_{2m+1},  dL/dA(t2) = w1 dL/da_{2m} + w2 dL/da_{2m+1}
 * (and the same for B with b_s).
 *   boundaries: DEVICE, the 2*steps states written by cheb_magnus4.
 *   grad: DEVICE in/out (in: dL/dpsi_T; out: dL/dpsi_0). grad_dt (steps), grad_nodes
 *   (4*steps), grad_h (n), grad_J (n*n): HOST, nullable.
 * Workspace and errors: as cheb_anneal_general_adjoint (cheb_adjoint_workspace_bytes).
 */
cheb_status_t cheb_magnus4_adjoint(int n, const double* h, const double* J, int steps, const double* dt,
                                   const double* nodes, const void* boundaries, const void* psi_T, void* grad,
                                   cheb_precision_t precision, double tol, cheb_method_t method, double* grad_dt,
                                   double* grad_nodes, double* grad_h, double* grad_J, void* workspace,
                                   size_t workspace_bytes, void* stream);

/*
 * psi <- psi(T) under H(t) = A(t) sum_j X_j + B(t) H_P with the number of equal Magnus
 * steps chosen a posteriori (the paper selects steps from an O(1) error term whose
 * constants it does not print; this is the step-doubling estimate instead): runs of
 * steps0 and 2*steps0 steps estimate the integration error of the second as
 * ||y_M - y_2M|| / 15 (fourth order), and if that exceeds tol a last run uses
 * ceil(2 steps0 (estimate / tol)^(1/4) * 1.1) steps. Each exponential's series uses the
 * precision's default budget (2^-23 for FP32, 1e-12 for FP64).
 *   schedule, user: the schedule, sampled through cheb_magnus4_nodes.
 *   steps_used: HOST out, the step count of the returned state. err_estimate: HOST out
 *   (nullable), the estimate scaled to that step count.
 * Workspace: cheb_magnus4_adaptive_workspace_bytes(n, precision) (the expmv workspace
 * plus two state vectors). Synchronises the stream once. Errors: as cheb_magnus4.
 */
size_t cheb_magnus4_adaptive_workspace_bytes(int n, cheb_precision_t precision);
cheb_status_t cheb_magnus4_adaptive(int n, const double* h, const double* J, double T, cheb_schedule_fn schedule,
                                    void* user, int steps0, double tol, void* psi, cheb_precision_t precision,
                                    cheb_method_t method, void* workspace, size_t workspace_bytes, void* stream,
                                    int* steps_used, double* err_estimate);

/*
 * Batched independent instances (Sec. III.A batches many small problems per launch):
 * psi_i <- exp(-i t_i H_i) psi_i for i = 0..B-1, each with its own n_i, couplings,
 * gamma_i and t_i, and its own spectral interval and polynomial (the paper pads the
 * batch to the largest radius instead).
 *   n:        HOST array of B sizes (1..33).
 *   offsets:  HOST array of B element offsets of each state in psi_cat (complex
 *             elements of the given precision; each state must start 16-byte aligned).
 *   h_cat:    HOST, the h vectors concatenated (sum n_i doubles).
 *   J_cat:    HOST, the n_i x n_i row-major J matrices concatenated (sum n_i^2 doubles).
 *   gamma, t: HOST arrays of B doubles.   psi_cat: DEVICE, in/out.
 *   workspace: cheb_batched_workspace_bytes(B, n, precision) bytes (256-aligned).
 *   infos:    nullable HOST array of B cheb_info_t; requesting it synchronises.
 * The spectral bounds of all instances need one synchronisation of the stream.
 * FP32 instances run in one persistent launch (cheb_set_batch_persistent); otherwise
 * instances with n <= 13 (FP32) or n <= 12 (FP64) run together in one launch, the next
 * four sizes on thread-block clusters, larger ones on an internal pool of streams
 * joined back into `stream`.
 * Errors: as cheb_expmv.
 */
size_t cheb_batched_workspace_bytes(int B, const int* n, cheb_precision_t precision);
/* FP32 batches run as one persistent cooperative launch: one CTA per SM takes work slots
 * from a counter, longest instance first; n <= 12 runs whole in one CTA's shared memory,
 * larger n on a team of 1..64 CTAs (2^(n-14)) that steps through the Clenshaw
 * recurrence with the vectors in L2 and a bounded team barrier after every pass (a wait
 * that runs out reports CHEB_ERR_TIMEOUT). on = 1 (default) runs one CTA of 512
 * threads per SM; on = 2 two CTAs per SM with half the registers per thread; on = 0
 * selects the per-size launches and the stream pool described
 * above (process-wide; FP64 batches always use them). */
cheb_status_t cheb_set_batch_persistent(int on);
int cheb_get_batch_persistent(void);
cheb_status_t cheb_expmv_batched(int B, const int* n, const int64_t* offsets, const double* h_cat,
                                 const double* J_cat, const double* gamma, const double* t,
                                 void* psi_cat, cheb_precision_t precision, double tol,
                                 cheb_method_t method, void* workspace, size_t workspace_bytes,
                                 void* stream, cheb_info_t* infos);

/*
 * Reverse-mode gradients (no counterpart in the paper; derived from Algorithm 2).
 * For a real loss L of the schedule's final state y and ybar = dL/dy in the
 * convention dL = Re<ybar, dy> (torch's for complex tensors; for L = |y|^2,
 * ybar = 2y), the adjoint of the Clenshaw recurrence gives
 *   bbar_0 = ybar, bbar_1 = Ht bbar_0, bbar_k = 2 Ht bbar_{k-1} - bbar_{k-2},
 *   psibar = sum_k conj(c_k) bbar_k,
 *   dL = Re sum_{k<K} w_k <bbar_k, dHt b_{k+1}>  (w_0 = 1, w_k = 2).
 * The forward vectors b_k of each segment are recomputed from its start state and
 * either all kept (workspace for K vectors) or regenerated upward from (b_1, b_2)
 * and reset from anchor pairs. The spectral interval (c, r) is held fixed (the
 * exact exp(-itH) does not depend on it); dL/dt_s uses the exact dy/dt = -i H y.
 * The gamma derivative uses Ht b_{k+1} = (b_k + b_{k+2} - c_k psi)/2, so no extra
 * operator applications are needed. The relative phase that round-off introduces
 * between the adjoint and the stored forward states is removed per segment from the
 * invariant <bbar_s, y_s> = <ybar_T, y_T>.
 *
 * cheb_adjoint_workspace_bytes(n, precision, store_vectors): workspace for
 *   cheb_anneal_adjoint with a pool of `store_vectors` state vectors. A segment of
 *   degree K keeps every b_k when store_vectors >= K; otherwise it needs
 *   store_vectors >= 8 (a ring of 6 plus (store_vectors - 6)/2 anchor pairs).
 *   store_vectors = 0 sizes the workspace of cheb_energy_grad.
 * cheb_anneal_adjoint:
 *   boundaries: DEVICE, the S segment-start states written by cheb_anneal.
 *   psi_T:      DEVICE, the final state.
 *   grad:       DEVICE in/out: in = ybar at the final state; out = psibar at the
 *               initial state.
 *   grad_gamma, grad_t (HOST, S doubles), grad_h (HOST, n), grad_J (HOST, n*n,
 *   strict upper triangle filled, rest zero): nullable outputs.
 *   S = 1 with boundaries = the input state is the gradient of one cheb_expmv.
 * cheb_energy_grad: L = <psi|H_P|psi> (FP64 reduction), grad_psi (DEVICE out) =
 *   2 H_P psi, grad_h, grad_J as above (HOST).
 * Errors: INVALID_ARG, WORKSPACE (too small, or a segment with K > store_vectors
 *   and store_vectors < 8), CUDA, TIMEOUT, UNSUPPORTED (time slicing needed).
 */
size_t cheb_adjoint_workspace_bytes(int n, cheb_precision_t precision, int store_vectors);
cheb_status_t cheb_anneal_adjoint(int n, const double* h, const double* J, int S, const double* gamma_s,
                                  const double* t_s, const void* boundaries, const void* psi_T,
                                  void* grad, cheb_precision_t precision, double tol,
                                  cheb_method_t method, double* grad_gamma, double* grad_t,
                                  double* grad_h, double* grad_J, void* workspace,
                                  size_t workspace_bytes, void* stream);
/*
 * The adjoint of cheb_anneal_general (segments H_s = b_s H_P + a_s sum_j X_j): as
 * cheb_anneal_adjoint, plus dL/db_s = sum_z G_s(z) E(z) / r_s with G_s = dL/dDt on the
 * segment and r_s its (frozen) radius; dh, dJ collect b_s / r_s times the moments of
 * each G_s. boundaries are the segment starts written by cheb_anneal_general.
 *   grad_a, grad_b, grad_t: HOST, S doubles each (nullable); other arguments as
 *   cheb_anneal_adjoint (same workspace).
 */
cheb_status_t cheb_anneal_general_adjoint(int n, const double* h, const double* J, int S,
                                          const double* a_s, const double* b_s, const double* t_s,
                                          const void* boundaries, const void* psi_T, void* grad,
                                          cheb_precision_t precision, double tol, cheb_method_t method,
                                          double* grad_a, double* grad_b, double* grad_t, double* grad_h,
                                          double* grad_J, void* workspace, size_t workspace_bytes,
                                          void* stream);
/*
 * Forward runs that leave the adjoint's checkpoints behind (no counterpart in the
 * paper). They compute the same schedule as cheb_anneal / cheb_anneal_general, but
 * run the last segment on the adjoint's step runner and keep its Clenshaw vectors
 * b_K .. b_1 in the pool of an ADJOINT workspace (every b_k when the pool holds K
 * vectors, else the ring and anchor pairs). The next cheb_anneal_adjoint /
 * cheb_anneal_general_adjoint call with the same workspace (pointer and size), the
 * same n, S, schedule, couplings, precision, tol and method, psi_T = this psi and the
 * same boundaries then skips that segment's forward recomputation; for S = 1 (one
 * exp(-itH) psi) that is one of its three passes over the Clenshaw recurrence.
 *   psi:        DEVICE in/out, as cheb_anneal (out = the final state psi_T).
 *   boundaries: DEVICE, required: receives the S segment-start states.
 *   workspace:  cheb_adjoint_workspace_bytes(n, precision, store_vectors) bytes,
 *               256-byte aligned; between this call and the adjoint only forward
 *               entry points may use it (they touch its leading forward workspace,
 *               not the pool).
 * Any adjoint call on the workspace consumes the checkpoint; arguments that differ
 * make the adjoint recompute the segment (the result is the same either way). The
 * record is kept on the host per workspace pointer.
 * Errors: as cheb_anneal_adjoint (WORKSPACE when the pool is too small for the last
 * segment, UNSUPPORTED when it needs time slicing).
 */
cheb_status_t cheb_anneal_checkpointed(int n, const double* h, const double* J, int S,
                                       const double* gamma_s, const double* t_s, void* psi,
                                       cheb_precision_t precision, double tol, cheb_method_t method,
                                       void* boundaries, void* workspace, size_t workspace_bytes,
                                       void* stream);
cheb_status_t cheb_anneal_general_checkpointed(int n, const double* h, const double* J, int S,
                                               const double* a_s, const double* b_s,
                                               const double* t_s, void* psi,
                                               cheb_precision_t precision, double tol,
                                               cheb_method_t method, void* boundaries,
                                               void* workspace, size_t workspace_bytes,
                                               void* stream);
cheb_status_t cheb_energy_grad(int n, const double* h, const double* J, const void* psi,
                               void* grad_psi, cheb_precision_t precision, double* energy,
                               double* grad_h, double* grad_J, void* workspace,
                               size_t workspace_bytes, void* stream);

/* Same as cheb_expmv with an explicit kernel path (cheb_path_t), optionally OR-ed
 * with CHEB_FLAG_EVAL_BOUND; used to time the plain one-pass GPU path against the
 * fused path and to request the evaluation bound. */
cheb_status_t cheb_expmv_path(int n, const double* h, const double* J, double gamma, double t,
                              void* psi, cheb_precision_t precision, double tol,
                              cheb_method_t method, int time_splits, int path, void* workspace,
                              size_t workspace_bytes, void* stream, cheb_info_t* info);

/*
 * Bit split of the fused FP32 step for n qubits (n >= 11). Each Clenshaw step
 * needs all n bit-flip partners of every amplitude (Sec. II.D); the fused step
 * takes bits [0, 11) from a shared-memory tile and bits [11, 11 + l) from partner
 * tiles through L2 in one pass, and the remaining h bits in strided passes of 3..9
 * bits each (at most four), with 11 + l + h = n, 0 <= l <= 6, h = 0 or h >= 3.
 * cheb_set_fused_split overrides the built-in choice for this n (process-wide,
 * all devices); l = -1 restores the default. cheb_get_fused_split reports the
 * split that the next call at this n will use.
 * Errors: INVALID_ARG for an impossible split or n outside 11..33.
 */
cheb_status_t cheb_set_fused_split(int n, int l, int h);
cheb_status_t cheb_get_fused_split(int n, int* l, int* h);

/*
 * Bit split of the fused float-float step of the FP64 path for n qubits (n >= 11): bits
 * [0, 10) from a shared-memory tile of 1024 complex amplitudes, bits [10, 10 + l) from
 * L2 partner tiles, and the remaining h bits in strided passes of 6..9 bits (5..8 bits
 * on rows of 16 amplitudes where rows lie at least 2 MB apart), at most four, with
 * 10 + l + h = n, 0 <= l <= 6. Same conventions as cheb_set_fused_split.
 * Errors: INVALID_ARG for an impossible split or n outside 11..33.
 */
cheb_status_t cheb_set_fused_split_fp64(int n, int l, int h);
cheb_status_t cheb_get_fused_split_fp64(int n, int* l, int* h);

/*
 * L2-blocked step tail of the fused FP32 step (Sec. II.D matvec, scheduled for a
 * 126 MB L2; no counterpart in the paper). When on, the last strided pass and the low
 * pass of each step run as one persistent launch: amplitudes are grouped by their
 * bits [11, lo) (lo = first bit of the last strided range), and the low tiles of
 * a group are processed right after the strided tiles of that group, so b_{k+1}
 * and the partial sum are read back from L2 instead of DRAM. Results are identical
 * to the separate launches (same operations in the same order per amplitude).
 * Used for n >= 22 when the split has at least two strided passes, l <= 1 and a
 * last range of 6..9 bits; other splits keep the separate launches.
 * Mode 2 blocks the two strided passes of a split that has exactly two (ranges
 * A = [loA, loB) and B = [loB, n) of 6..9 bits, B no wider than A and at most one bit
 * narrower), in the FP32 step and in the float-float step of the FP64 path (n >= 22):
 * amplitudes are grouped by their bits above a 128-byte row and below loA, and the
 * tiles of the upper range B of a group run right after the tiles of range A of that
 * group, so b_{k+1} and the partial sum come back from L2: the two passes move half
 * the DRAM bytes of two separate passes (24 B per amplitude in FP32). Flip sums are plain FP32 in descending bit
 * order, as in the separate launches, so results are identical. The lag between a
 * group's A and B tiles keeps about 48 MB of the two vectors live in L2 (one group of
 * 32 MB, two of 16 MB); the environment variable CHEB_PAIR_LAG (1..16) overrides it.
 * on: 0 off, 1 the blocked tail (FP32 only), 2 the blocked strided pair, -1 automatic
 * (the default: the blocked strided pair from n = 26 on for FP32 and from n = 28 on for
 * FP64, separate launches below).
 * Process-wide; the autotuner's per-(precision, n) choice takes precedence.
 * cheb_get_fused_blocking returns the setting.
 */
cheb_status_t cheb_set_fused_blocking(int on);
int cheb_get_fused_blocking(void);

/*
 * Compensated flip sums in the fused FP32 step (the bit-flip sum of the matrix-free
 * matvec, Sec. II.D, whose rounding is the sqrt(d) gamma_d term of the evaluation
 * bound, Sec. II.B.3). When on, each pass adds its flip terms with Kahan's
 * compensated summation instead of plain FP32 adds; the partial sums of different
 * passes are still combined in FP32. on: 0 off (default), 1 on (process-wide).
 */
cheb_status_t cheb_set_fused_compensated(int on);
int cheb_get_fused_compensated(void);

/*
 * Autotuner of the Clenshaw step configuration (no counterpart in the paper). For
 * (n, precision) it times, on the calling device and the given stream, `steps`
 * Clenshaw steps of a synthetic problem of that size under the built-in choice and
 * under every candidate: the plain one-pass kernel (n <= 24 FP32, <= 26 FP64) and the
 * fused step with each valid bit split of at most 4 (FP32) or 5 (FP64) L2 partner
 * bits, and for FP32 the L2-blocked tail and strided pair where the split allows them. The fastest
 * candidate is installed process-wide: AUTO then uses that path, split and blocking
 * for n (cheb_set_fused_split / cheb_set_fused_split_fp64 override it again).
 * If the environment variable CHEB_AUTOTUNE_CACHE names a file, the result is appended
 * to it as a line "cheb-tune-1 <device name> <prec> <n> <path> <l> <h> <blocking> <ms>",
 * and the first Clenshaw run of a process applies the lines recorded for its device.
 *   steps: 2..64 timed steps per candidate (each candidate runs twice, the second timed).
 *   workspace: cheb_autotune_workspace_bytes(n, precision) bytes (the expmv workspace
 *   plus one state vector). Synchronises the stream once per candidate.
 *   result: HOST out.
 * Errors: INVALID_ARG (n < 14 FP32 or < 13 FP64, steps outside 2..64, null result),
 * WORKSPACE, CUDA, TIMEOUT.
 */
typedef struct {
    int path;                    /* CHEB_PATH_PLAIN or CHEB_PATH_FUSED */
    int l, h;                    /* the split, for FUSED */
    int blocking;                /* FP32: 1 L2-blocked step tail, 2 L2-blocked strided pair */
    int candidates;              /* configurations timed */
    double best_ms_per_step;     /* the chosen configuration */
    double default_ms_per_step;  /* the built-in choice */
} cheb_tune_result_t;
size_t cheb_autotune_workspace_bytes(int n, cheb_precision_t precision);
cheb_status_t cheb_autotune(int n, cheb_precision_t precision, int steps, void* workspace, size_t workspace_bytes,
                            void* stream, cheb_tune_result_t* result);
/* Applies the lines of an autotuner cache file recorded for `device` (a device name
 * with spaces replaced by '_'; NULL = the current device, which needs a GPU). applied:
 * HOST out (nullable), the number of lines applied. Host only otherwise.
 * Errors: INVALID_ARG (null path, file not readable). */
cheb_status_t cheb_autotune_load(const char* path, const char* device, int* applied);
/* Drops every tuned choice and split override (the built-in choices apply again). */
cheb_status_t cheb_autotune_reset(void);

/*
 * General polynomial p(Ht) psi (Algorithm 2 with caller-supplied coefficients):
 * psi <- sum_{m=0}^{K} c_m T_m(Ht) psi with Ht = (H - center) / radius and
 * H = diag(E) + gamma * sum_j X_j. The caller chooses center and radius (radius > 0);
 * the series is only meaningful when ||Ht|| <= 1 (radius >= the value cheb_expmv uses).
 *   coeffs: HOST array of 2*(K+1) doubles (re, im), 0 <= K <= 65536.
 * Errors: INVALID_ARG, WORKSPACE, CUDA, UNSUPPORTED.
 */
/*
 * Monomial to Chebyshev basis (the two bases of Sec. II.B): given
 * p(x) = sum_{m=0}^{K} a_m x^m, writes c with p(x) = sum_{k=0}^{K} c_k T_k(x), so that
 * cheb_poly_apply evaluates a polynomial given in the monomial basis by the Clenshaw
 * recurrence. Exact up to rounding (computed in long double, O(K^2)).
 *   monomial, chebyshev: HOST arrays of 2*(K+1) doubles (re, im); may not alias.
 * Errors: INVALID_ARG (K < 0 or > 65536, null pointers, non-finite input).
 */
cheb_status_t cheb_monomial_to_chebyshev(int K, const double* monomial, double* chebyshev);

cheb_status_t cheb_poly_apply(int n, const double* h, const double* J, double gamma,
                              double center, double radius, int K, const double* coeffs,
                              void* psi, cheb_precision_t precision, int path, void* workspace,
                              size_t workspace_bytes, void* stream);

/*
 * <psi|H_P|psi> and ||psi||^2 in FP64 on the device (Ising diagonal recomputed from
 * the couplings). Synchronises the stream. energy, norm2: HOST outputs.
 */
cheb_status_t cheb_energy(int n, const double* h, const double* J, const void* psi,
                          cheb_precision_t precision, void* workspace, size_t workspace_bytes,
                          void* stream, double* energy, double* norm2);

/*
 * Instrumentation (no counterpart in the paper; used to attribute time).
 * cheb_launch_count: number of kernels this library has launched in this process
 *   (all devices, monotone).
 * cheb_profile_enable(1): from now on, bracket every Clenshaw step kernel and
 *   every adjoint accumulation kernel with a pair of CUDA events on its stream (a
 *   few microseconds of overhead per step).
 * cheb_profile_read(kind, count, total_ms): synchronises the recorded events and
 *   returns how many launches of that kind were timed and their summed device
 *   time. cheb_profile_reset drops the records.
 * Kinds: 3 plain one-pass step, 5 adjoint accumulation (cheb_anneal_adjoint),
 * 6 fused low pass, 7 fused strided (high-bit) pass, 8 L2-blocked step tail (last
 * strided pass + low pass, cheb_set_fused_blocking(1)), 9 L2-blocked strided pair
 * (cheb_set_fused_blocking(2)).
 */
typedef enum {
    CHEB_KERNEL_STEP_PLAIN = 3,
    CHEB_KERNEL_ADJOINT_ACC = 5,
    CHEB_KERNEL_FUSED_LOW = 6,
    CHEB_KERNEL_FUSED_HIGH = 7,
    CHEB_KERNEL_FUSED_TAIL = 8,
    CHEB_KERNEL_FUSED_PAIR = 9
} cheb_kernel_kind_t;

/*
 * Failure-detection self-test (no counterpart in the paper). Every device-side wait of
 * this library is bounded: it gives up after about 2 s, records a timeout in the
 * workspace status word and lets the kernel return, and the call reports
 * CHEB_ERR_TIMEOUT. This entry point runs both kinds of wait, each with a ~1 ms limit,
 * on a wait that nothing satisfies (an mbarrier that nothing arrives on, as in the TMA
 * kernels; a team barrier whose teammate never comes, as in the persistent batch
 * kernel), and returns CHEB_ERR_TIMEOUT when both reported their timeout (the expected
 * answer; CHEB_OK otherwise). The context stays usable afterwards.
 *   workspace: DEVICE, at least 16 bytes, 4-byte aligned. Synchronises.
 */
cheb_status_t cheb_wait_selftest(void* workspace, size_t workspace_bytes, void* stream);

/*
 * Host check of the blocked strided pair's work order (no counterpart in the paper; the
 * pair is this library's L2 blocking of the strided passes of the Clenshaw step,
 * Sec. II.D). For 2^gbits groups, ranges of HA and HB bits (1..9) and a lag of
 * 1..2^gbits groups, the item indices handed out by the pair's global counter must
 * name every A-tile (2^HB per group) and every B-tile (2^HA per group) exactly once,
 * followed by the end marker, with every B-tile of a group after all of that group's
 * A-tiles: a B-tile's wait for its group then only depends on items taken before it.
 * Returns 0 when all of this holds (min_gap, if not NULL, receives the smallest index
 * distance between a group's last A-tile and its first B-tile), 1 for an item out of
 * range, 2 for an item handed out twice, 3 for a missing one, 4 for a B-tile before its
 * group's last A-tile, 5 for a misplaced end marker, -1 for invalid arguments
 * (gbits 0..16). Host only; no device or stream is used.
 */
int cheb_pair_schedule_check(int gbits, int HA, int HB, int lag, long long* min_gap);

/*
 * Device-side status of a workspace (no counterpart in the paper). A call made
 * without an info struct does not synchronise, so a bounded wait that ran out during
 * it is not in its return value; the condition stays recorded in the workspace's
 * status word until the next call on that workspace starts. This entry point
 * synchronises the stream, returns CHEB_ERR_TIMEOUT (a wait ran out), CHEB_ERR_CUDA (a
 * launch was refused inside a kernel) or CHEB_OK, and clears the word. Valid for the
 * workspaces of cheb_expmv, cheb_expmv_path, cheb_poly_apply, cheb_anneal,
 * cheb_anneal_general, cheb_magnus4 and the adjoint entry points.
 *   workspace: DEVICE, the workspace of the call to query (256-byte aligned).
 */
cheb_status_t cheb_workspace_status(void* workspace, size_t workspace_bytes, void* stream);

/*
 * Programmatic dependent launch of the fused step kernels (no counterpart in the paper):
 * when on (the default), each pass is launched so that its CTAs may be scheduled while
 * the previous pass drains; a kernel waits for its predecessor's completion (and memory)
 * before it reads any vector the predecessor writes, so results are unchanged. Event
 * profiling (cheb_profile_enable) launches without it. on: 0 or 1 (process-wide).
 */
cheb_status_t cheb_set_programmatic_launch(int on);

long long cheb_launch_count(void);
cheb_status_t cheb_profile_enable(int on);
cheb_status_t cheb_profile_reset(void);
cheb_status_t cheb_profile_read(int kind, long long* count, double* total_ms);

#ifdef __cplusplus
}
#endif

#endif /* CHEB_EXPMV_H */
