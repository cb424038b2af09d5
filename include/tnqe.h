/*
 * tnqe.h -- C ABI of the GB300 (sm_103a) matrix-element library for the
 * tensor-network quantum eigensolver of Leimkuhler & Whaley, arXiv 2404.10223.
 *
 * The wavefunction is a linear combination of M matrix product states (MPS),
 * each in its own orbital basis (Eq. 8, Sec. II B).  The library fills the
 * subspace matrices H_ij = <psi_i|H|psi_j> and S_ij = <psi_i|psi_j> (Eq. 10)
 * for a list of pairs and solves H c = E S c (Eq. 9) by canonical
 * orthogonalisation (Sec. IV C, App. A2).
 *
 * Conventions (fixed by this ABI):
 *  - Spatial-orbital sites, local dimension d = 4, local index
 *    k = n_alpha + 2 n_beta (Sec. II A lists vac, up, down, updown as
 *    00, 01, 10, 11).  |k_0 ... k_{N-1}> = prod_p (a+_{p,alpha})^{n}(a+_{p,beta})^{n} |vac>
 *    with p ascending; Jordan-Wigner order 0a, 0b, 1a, 1b, ...
 *  - Hamiltonian (Eq. 1) in chemists' notation:
 *    H = sum_{pq,s} h_pq a+_ps a_qs + 1/2 sum_{pqrs,st} (pq|rs) a+_ps a+_rt a_st a_qs.
 *  - State j is psi_j = G(U_j) |MPS_j>, where G(V) a+_q G(V)^-1 = sum_p a+_p V_pq
 *    and column p of U_j is orbital p of basis j in the reference orbitals.
 *  - Pair (i, j) brings MPS_j into basis i with the Givens network of
 *    V = U_i^T U_j (Eq. 11) and SVD truncation, then contracts
 *    <MPS_i| H^(i) |G(V) MPS_j> against the MPO of H expressed in basis i.
 *
 * Memory: all input arrays are copied; the caller keeps ownership.  Output
 * arrays may live in host or device memory (detected per pointer).  Every
 * call returns a status; no exception, exit or abort crosses the ABI.  A
 * context is not thread-safe: use one context per host thread.
 */
#ifndef TNQE_H
#define TNQE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tnqe_ctx tnqe_ctx;

typedef enum {
  TNQE_OK = 0,
  TNQE_ERR_ARG = 1,      /* invalid argument (sizes, non-orthogonal U, broken MPS form) */
  TNQE_ERR_STATE = 2,    /* call out of order (e.g. unknown MPS id) */
  TNQE_ERR_NOMEM = 3,    /* device or host allocation failed */
  TNQE_ERR_CUDA = 4,     /* a CUDA runtime call failed */
  TNQE_ERR_NOCONV = 5,   /* a Jacobi iteration hit its sweep limit (results still written) */
  TNQE_ERR_TIMEOUT = 6,  /* a bounded device wait gave up */
  TNQE_ERR_NUMERIC = 7   /* NaN/Inf in an output */
} tnqe_status;

/* Contraction precision.  The rotation SVDs and the solve are FP64 always.
 * TF32X3: FP32 environments; GEMM operands split into TF32 high and low parts,
 *   three products (hi.hi + hi.lo + lo.hi) accumulated in FP32 on the tensor cores;
 *   stage 2 in FP32.  About 21 bits per operand, FP32 rounding in every sum.
 * BF16X3 / BF16X6 / BF16X10 / BF16X15: double-float environments (two FP32
 *   values, about 48 bits); every GEMM operand row is scaled by a power of two
 *   and split into S = 2 / 3 / 4 / 5 fixed-point BF16 slices of 8 bits each; the
 *   3 / 6 / 10 / 15 slice products of order <= S + 1 run on the tensor cores with
 *   FP32 accumulation that is exact for the three leading products (integer
 *   multiples of a power of two, bounded by 2^24 for K <= 1024); stage 2 in
 *   double-float arithmetic.  The error is the slicing truncation alone:
 *   about 2^-16, 2^-24, 2^-32, 2^-40 of the row maxima.  Bond dimensions above 256
 *   return TNQE_ERR_ARG in these modes. */
typedef enum {
  TNQE_PREC_FP64 = 0,
  TNQE_PREC_TF32X3 = 1,
  TNQE_PREC_BF16X3 = 2,
  TNQE_PREC_BF16X6 = 3,
  TNQE_PREC_BF16X10 = 4,
  TNQE_PREC_BF16X15 = 5
} tnqe_precision;

typedef struct {
  int precision;            /* tnqe_precision; the rotation SVDs and the solve are FP64 always */
  int chi_rot;              /* bond-dimension cap of a rotated state; 0 = max bond dim of MPS j */
  double cutoff;            /* keep sigma_l > cutoff * sigma_1 (relative singular-value threshold) */
  double solve_eps;         /* keep eigenvalues of S above solve_eps * lambda_max */
  int renormalize_rotated;  /* 1: rescale a rotated state to its pre-rotation norm (App. A1) */
  int max_jacobi_sweeps;    /* Jacobi sweep limit (SVD and eigensolver) */
  long long max_spin;       /* iteration limit of any device-side wait */
  void* cuda_stream;        /* cudaStream_t to launch on; NULL = a stream owned by the context */
  int device;               /* CUDA device ordinal */
  int use_graphs;           /* 1: replay repeated tnqe_matrix_elements calls from a captured CUDA graph */
  int contraction_form;     /* tnqe_form: FP64 contraction in charge blocks (default) or dense */
  const char* autotune_cache; /* file of tuned launch shapes per pair-list class (NULL = none); copied */
  long long workspace_limit;  /* contraction workspace bytes per wave; 0 = 60 % of free device memory */
} tnqe_options;

/* Form of the FP64 contraction (TNQE_PREC_FP64; the split-precision modes are dense).
 * BLOCKS: every bond index has a particle-number charge (n_alpha, n_beta) and every
 *   MPO channel the charge change of its operator string (particle number and S_z
 *   are conserved, Sec. II C / Sec. IV A), so an environment entry L[a][w][b] can
 *   be nonzero only when q(a) = q(b) + d(w).  Only those blocks are computed.
 * DENSE: the same contraction over the zero-padded dense tensors (the masked
 *   zeros are multiplied); the plain reference form. */
typedef enum {
  TNQE_FORM_BLOCKS = 0,
  TNQE_FORM_DENSE = 1
} tnqe_form;

/* Fill *opt with defaults: FP64, chi_rot 0, cutoff 1e-14, solve_eps 1e-10,
 * no renormalisation, 60 Jacobi sweeps, max_spin 1<<26, own stream, device 0,
 * graphs on, charge-block contraction. */
void tnqe_default_options(tnqe_options* opt);

/* The nearest-neighbour Givens plan of a relative rotation V = U_i^T U_j
 * (Eq. 11, App. A3), as tnqe_matrix_elements applies it, computed on the
 * host.  V: N*N row-major orthogonal.  Gate g acts on sites (site[g],
 * site[g] + 1) as G(J^T), J = [[c, -s], [s, c]] at rows/columns (site,
 * site + 1); side[g] = 0 puts the singular values into the left tensor, 1 into
 * the right.  Gates come in application order, N(N-1)/2 of them; cap is the
 * capacity of site, side, c, s (TNQE_ERR_ARG if smaller).  *neg_site is the
 * orbital whose creators change sign (det V = -1), else -1.  No GPU needed. */
tnqe_status tnqe_givens_host(const double* V, int N, int* site, int* side, double* c, double* s, int cap,
                             int* ngates, int* neg_site);

/* The 16 x 16 two-site gate G(J^T) of one Givens rotation, J = [[c, -s], [s, c]]
 * (c^2 + s^2 = 1), on the local states k = n_alpha + 2 n_beta of the two
 * sites: G[(4 k1' + k2') * 16 + (4 k1 + k2)], the matrix the rotation kernel
 * applies.  No GPU needed. */
tnqe_status tnqe_gate_host(double c, double s, double* G);

/* h' = U^T h U and (pq|rs)' = sum U_ap U_bq U_cr U_ds (ab|cd): the integrals in
 * basis U (column p of U = orbital p), as tnqe_add_mps uses them for the MPO of
 * a state.  h_out N*N, eri_out N^4 (row-major, caller's host memory). */
tnqe_status tnqe_rotate_integrals_host(const double* h1, const double* eri, const double* U, int N, double* h_out,
                                       double* eri_out);

/* The checks tnqe_add_mps makes on a state, on the host, no GPU needed:
 * tensors / bond_dims / U as for tnqe_add_mps, for N orbitals and
 * (n_alpha, n_beta) electrons.  Returns TNQE_OK, or TNQE_ERR_ARG with the
 * reason in msg (msg_len bytes including the terminating zero; msg may be
 * NULL): U not orthogonal to 1e-12, bond dimensions outside [1, 256] or not
 * 1 at the ends, a bond index with no weight, an entry that breaks the
 * particle-number block structure, a state outside the (n_alpha, n_beta)
 * sector, or a site 0..N-2 that is not left-orthonormal to 1e-10. */
tnqe_status tnqe_check_mps(int N, int n_alpha, int n_beta, const double* const* tensors, const int* bond_dims,
                           const double* U, char* msg, int msg_len);

/* The Hamiltonian MPO the library builds for integrals (h1, eri) (Eq. 1 in
 * second quantisation, Sec. II A; one per state basis inside tnqe_add_mps),
 * computed on the host, no GPU needed.  h1: N*N row-major; eri: N^4
 * row-major chemists' (pq|rs); 1 <= N <= 32.  Site t is a sparse
 * (4 D_{t+1}) x (4 D_t) matrix in CSR: row k * D_{t+1} + w' (bra local state
 * k, right channel w'), column w * 4 + k' (left channel w, ket local state
 * k'); channel 0 of every bond is the identity string, channel 1 of bonds
 * >= 1 the completed Hamiltonian, so D_0 = 1 and D_N = 2.
 * Outputs: dims[N + 1] (bond dimensions D_t), nnz[N] (nonzeros per site).
 * If rowptr, col and val are all non-NULL they receive every site in turn:
 * rowptr holds sum_t (4 D_{t+1} + 1) entries (site-local offsets), col and
 * val hold sum_t nnz[t] entries; cap is the capacity of col and val
 * (TNQE_ERR_ARG if it is too small).  Call once with NULL buffers to size
 * them.  The result does not depend on the machine (fixed work shares). */
tnqe_status tnqe_mpo_host(const double* h1, const double* eri, int N, int* dims, long long* nnz, int* rowptr,
                          int* col, double* val, long long cap);

/* Create a context for N spatial orbitals and (n_alpha, n_beta) electrons.
 * h1: N*N row-major, symmetric.  eri: N^4 row-major (pq|rs).  Both copied.
 * Requires 1 <= N <= 32 and n_alpha, n_beta <= 14.  opt may be NULL.
 * On success *out owns all device memory of the context. */
tnqe_status tnqe_create(const double* h1, const double* eri, int N, int n_alpha, int n_beta,
                        const tnqe_options* opt, tnqe_ctx** out);

/* Add one state (Eq. 3).  tensors[s] points to site s, shape
 * [bond_dims[s]][4][bond_dims[s+1]] row-major FP64 (host memory).
 * bond_dims has N+1 entries, bond_dims[0] = bond_dims[N] = 1.
 * U: N*N row-major orthogonal (|U^T U - I|_max < 1e-12).
 * The MPS must be left-orthonormal on sites 0..N-2 (canonical centre on the
 * last site, Eq. A3) to 1e-10, and every bond index must carry a definite
 * (n_alpha, n_beta) charge: A[l,k,r] may be nonzero (above 1e-12 of the
 * site's largest entry) only when q(l) + q(k) = q(r), with the last bond at
 * (n_alpha, n_beta).  Violations return TNQE_ERR_ARG.  Uploads the tensors
 * (synchronously).  The Hamiltonian MPO in basis U is built on a host thread
 * that the first call needing it starts: tnqe_matrix_elements with this state
 * as a bra starts the build after enqueueing its rotations, waits for it while
 * the rotation kernel runs, and uploads the MPO (an error of the build is
 * reported by that call). */
tnqe_status tnqe_add_mps(tnqe_ctx* ctx, const double* const* tensors, const int* bond_dims,
                         const double* U, int* mps_id);

/* Drop every state and free its device buffers (waits for the context's
 * stream and for any MPO build still running). */
tnqe_status tnqe_reset_mps(tnqe_ctx* ctx);

/* Rotate MPS j into basis i (Eq. 11 with truncation, Sec. II D) and keep the
 * result for tnqe_get_rotated.  *discarded_weight (host, may be NULL) gets the
 * sum of squared discarded singular values over all gates. */
tnqe_status tnqe_rotate(tnqe_ctx* ctx, int i, int j, double* discarded_weight);

/* Copy the state kept by the last tnqe_rotate to host memory.  bond_dims gets
 * N+1 ints; tensors gets the sites back to back ([chi_s][4][chi_{s+1}] each)
 * and must hold max_doubles values; returns TNQE_ERR_ARG if it is too small. */
tnqe_status tnqe_get_rotated(tnqe_ctx* ctx, int* bond_dims, double* tensors, long long max_doubles);

/* H_ij and S_ij (Eq. 10) for npairs pairs.  pairs: 2*npairs ints (host),
 * (i, j) in either order: state i is the bra (the contraction runs in basis
 * i) and state j the rotated ket.  Without truncation H_ij = H_ji; with it
 * the two orders differ by the truncation error, so a caller assembling a
 * symmetric matrix picks one order per pair and keeps it (tnqe_solve reads
 * the upper triangle).  H_out, S_out: npairs doubles each, host or device.
 * Every pair is recomputed (rotation and contraction) on each call.
 *
 * One call puts all pairs' rotations (one launch) and contractions (a few
 * launches per site, every pair batched in each) on the stream without any
 * host synchronisation in between: rotated states are written at their bond
 * capacities min(chi_rot, full sector dimension), zero-padded, so the
 * contraction is planned before the truncation has run.  With use_graphs set,
 * the second call for a (pair list, states, options) combination also captures
 * that launch sequence into a CUDA graph; later identical calls replay it
 * (re-uploading their descriptors, then one cudaGraphLaunch).  Adding or
 * resetting states, changing options, or any workspace reallocation drops the
 * graphs.  If the workspace of all pairs does not fit in 60% of free device
 * memory (or in options.workspace_limit) the pairs run in waves that reuse the
 * workspace; in the FP64 charge-block form the waves follow each other in
 * stream order (no host synchronisation, captured and replayed like one wave),
 * in the other forms the host synchronises between waves and the call is not
 * captured.  In the BF16X* precisions and the charge-block FP64 form the pairs
 * (i, i), which need no rotation, are contracted on a second stream owned by the context (lowest
 * priority) while the rotation kernel runs on the context's stream; that
 * stream forks from and joins back into the context's stream within the call,
 * so work the caller orders after the call on its stream sees every result. */
tnqe_status tnqe_matrix_elements(tnqe_ctx* ctx, const int* pairs, int npairs,
                                 double* H_out, double* S_out);

/* Launch-shape autotuner of the contraction: the CTA sizes (64, 128, 256) of
 * the three charge-block stages (FP64, charge-block form), or the stage-1 and
 * stage-3 GEMM N tiles (128 or 64 columns) and the MPO kernel width (8, 4, 2
 * ket columns per CTA) of the sliced BF16X* modes; a no-op for the other forms.
 * The pair list -- normally the one that will be computed repeatedly -- is
 * reduced to its class: N (which fixes the MPO bond dimensions), precision,
 * form and the multiset of (bra bond dimension, ket bond dimension) over its
 * pairs.  With
 * options.autotune_cache set, a class found in that file takes its stored
 * shapes without timing; otherwise three candidates are timed (each run twice,
 * the first warms allocations), each kernel keeps the shape with the smallest
 * summed device time, and the result is appended to the file as the line
 * "tnqe-tune <class> | bs_t1 bs_t2 bs_t3 bn1 bn3 spmm_bw".  Captured graphs
 * are dropped.  config (3 ints, may be NULL) gets the chosen shapes of the
 * active form; times (9 doubles, may be NULL) the per-candidate stage-1,
 * stage-3 and stage-2 milliseconds (zero when the cache supplied the shapes). */
tnqe_status tnqe_autotune(tnqe_ctx* ctx, const int* pairs, int npairs, int* config, double* times);

/* Set the CTA sizes of the three charge-block stages directly (64, 128 or 256). */
tnqe_status tnqe_set_block_tuning(tnqe_ctx* ctx, int t1, int t2, int t3);

/* Set the launch shapes directly: bn1, bn3 in {64, 128}; spmm_bw in
 * {0 (largest that fits), 1, 2, 4, 8}. */
tnqe_status tnqe_set_tuning(tnqe_ctx* ctx, int bn1, int bn3, int spmm_bw);

/* Drop every captured graph of the context. */
tnqe_status tnqe_clear_graphs(tnqe_ctx* ctx);

/* Number of captured graphs the context holds (0 for NULL). */
int tnqe_graph_count(const tnqe_ctx* ctx);

/* Generalized eigenproblem H c = E S c (Eq. 9) for M <= 32 by canonical
 * orthogonalisation (projection method, Sec. IV C), on the GPU in FP64.
 * H, S: M*M row-major, host; the upper triangle (i <= j) is used.
 * E: M doubles, the rank_kept ascending eigenvalues first, the rest NaN.
 * C: M*M row-major, column k = eigenvector k (C^T S C = I), zero beyond rank.
 * kappa1 = |c_1|^2 / sqrt(E_1^2 + 1) (App. A2).  Outputs are host memory. */
tnqe_status tnqe_solve(tnqe_ctx* ctx, const double* H, const double* S, int M,
                       double* E, double* C, int* rank_kept, double* kappa1);

/* tnqe_solve with the eigenvalue threshold of S given per call: keep
 * eigenvalues above eps * lambda_max (0 <= eps < 1).  eps = solve_eps is
 * tnqe_solve; eps = sqrt(DBL_EPSILON) is the pseudo-inverse tolerance
 * sqrt(eps_mach) |S| the paper uses for its inversion variant (Sec. IV C):
 * both variants span the same eigenvectors of S and differ in this threshold. */
tnqe_status tnqe_solve_ex(tnqe_ctx* ctx, const double* H, const double* S, int M, double eps,
                          double* E, double* C, int* rank_kept, double* kappa1);

/* Linear-dependence residuals of a subspace (the discard test of Sec. IV C):
 * residuals[j] = S_jj - s_j^T (S_<j)^+ s_j, s_j = S[0:j, j], S_<j = S[0:j, 0:j],
 * the pseudo-inverse keeping eigenvalues above eps * lambda_max.  It is the
 * squared norm of state j's component outside the span of states 0..j-1
 * (residuals[0] = S_00).  A state whose residual falls below a threshold
 * (1e-3 in the paper's discussion) adds nothing new and may be discarded.
 * S: M*M row-major host, upper triangle used, M <= 32; residuals: M doubles (host). */
tnqe_status tnqe_dependence(tnqe_ctx* ctx, const double* S, int M, double eps, double* residuals);

/* Change the contraction precision (tnqe_precision) of later calls. */
tnqe_status tnqe_set_precision(tnqe_ctx* ctx, int precision);

/* Change the form of the FP64 contraction (tnqe_form) of later calls. */
tnqe_status tnqe_set_form(tnqe_ctx* ctx, int form);


/* Device time (ms) of the phases of the last tnqe_matrix_elements call,
 * measured with CUDA events on the context stream:
 * times[0] rotation, times[1] contraction, times[2] whole call.
 * launches: number of kernels that call launched. */
tnqe_status tnqe_last_timing(const tnqe_ctx* ctx, double* times, int* launches);

/* Per-kernel profile of the last tnqe_matrix_elements call (n values written,
 * n <= TNQE_PROFILE_LEN):
 * [0] rotation kernel ms, [1] stage-1 GEMM ms (X = L B), [2] stage-2 MPO ms,
 * [3] stage-3 GEMM ms (L' = A^T Y), [4] rotation algorithmic FLOPs
 * (two-site contraction + gate + 4mn^2 + 8n^3 per SVD block), [5] stage-1 FLOPs,
 * [6] stage-2 algorithmic bytes (X read once, Y written once; dense forms),
 * [7] stage-3 FLOPs, [8] stage-2 FLOPs (in the charge-block form the FLOPs of
 * the blocks computed, counted on the device), [9] kernels launched, [10] slicing kernels ms and
 * [11] slicing algorithmic bytes (BF16X* modes: source read once, slices
 * written once).  Times come from CUDA events on the context stream around
 * each launch and are summed over sites. */
#define TNQE_PROFILE_LEN 12
tnqe_status tnqe_last_profile(const tnqe_ctx* ctx, double* prof, int n);

/* ---------------------------------------------------------------------------
 * One Givens gate without any allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- programs whose
 * device memory is all handed out by their own pool reserved at start-up (a
 * serving process that owns the GPU's memory, where a library allocation would
 * fail or fragment that pool), and host loops that must not pay the latency
 * and implicit device synchronisation of cudaMalloc / cudaFree.  Everything
 * else in this header allocates through the context.
 *
 * Applies G(J^T), J = [[c, -s], [s, c]] on two neighbouring orbitals, to the
 * two-site tensor A . B and splits it again by a truncated SVD, exactly as one
 * step of tnqe_rotate:  A [chi_l][4][chi_m], B [chi_m][4][chi_r] in device
 * memory; q_l, q_m, q_r (host) give every bond index's charge
 * n_alpha * 16 + n_beta, each bond's indices grouped in ascending charge.
 * Keeps k = min(chi_max, #{sigma > cutoff * sigma_1}) (at least 1) singular
 * values; sigma_side 0 puts them into A_out, 1 into B_out.  Writes
 * A_out [chi_l][4][k] and B_out [k][4][chi_r] (device, capacity for
 * chi_max), the new bond's charges q_out[k] (host, may be NULL; ascending),
 * *k_out and *discarded (host; sum of the squared dropped singular values).
 * chi_l, chi_m, chi_r, chi_max must not exceed TNQE_NOALLOC_MAX_CHI
 * (TNQE_ERR_ARG otherwise, with the reason in err when err is not NULL).
 *
 * Its working storage is one static device array of
 * TNQE_NOALLOC_SCRATCH_BYTES (about 6.3 MiB) that every GPU loading this
 * library keeps until the process exits.  The first call on a device (and
 * the first after a device reset) looks up that array's address for the
 * current device and context (cudaGetSymbolAddress); make that first call
 * before any stream capture begins on the device.  All calls share the one
 * array and each starts by overwriting its header: calls that may overlap on
 * the GPU (other streams, other host threads) race and must be serialised by
 * the caller.  The call copies its 16 KiB parameter block to the device,
 * launches one kernel, copies the result header back into host memory and
 * synchronises `stream` (a cudaStream_t, NULL = legacy default stream)
 * before returning. */
#define TNQE_NOALLOC_MAX_CHI 128
#define TNQE_NOALLOC_SCRATCH_BYTES 6569984
tnqe_status tnqe_apply_gate_noalloc(const double* A, const double* B, int chi_l, int chi_m, int chi_r,
                                    const int* q_l, const int* q_m, const int* q_r, double c, double s,
                                    int sigma_side, int chi_max, double cutoff, int max_sweeps,
                                    double* A_out, double* B_out, int* q_out, int* k_out,
                                    double* discarded, void* stream, char* err, int err_len);

/* Human-readable description of the last error on this context. */
const char* tnqe_last_error(const tnqe_ctx* ctx);

/* Release the context and all its device memory. */
void tnqe_destroy(tnqe_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* TNQE_H */
