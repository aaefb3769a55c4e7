/*
 * cbc.h -- C ABI of the GB300 (sm_103a) implementation of the Cholesky-based
 * compression (CBC) that applies a tree tensor network operator (TTNO; an MPO on a
 * chain) to a tree tensor network state (TTNS; an MPS on a chain) and compresses the
 * result to a maximum bond dimension and/or a truncation tolerance.
 *
 * Method: arXiv 2601.19650, Sec. III.  Problem statement: Eq. (abstr_application),
 * |psi'> ~ O |psi>, with |psi> a TTNS (Sec. II A, Eq. (ttns)) and O a TTNO on the same
 * tree (Sec. II C, Eq. (ttno)).  The tensor-train sweeps follow Sec. III A
 * (Eqs. (tt_cbc_first_contraction), (right_sweep_init_contr), (tt_cbc_qr_decomp),
 * (tt_cbc_final_contraction)); trees follow Sec. III B (Eqs.
 * (cbc_tree_first_contraction) ... (cbc_final_contraction)).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Topology: n_nodes nodes; parent[i] is the parent of node i, -1 for exactly one root.
 * phys_dim[i] >= 1 is the physical dimension (1 = virtual node).  bond_dim[i] is the
 * dimension of the edge from i to its parent (ignored at the root, whose parent leg has
 * dimension 1).  A chain parent[i] = i-1 is a tensor train rooted at its first site,
 * the paper's imaginary-site-0 convention (Sec. II B).
 *
 * Leg order of node tensors (row-major, contiguous, children in ascending node id):
 *   state    T[i]: [parent, phys, child_0, child_1, ...]
 *   operator W[i]: [parent, phys_out, phys_in, child_0, child_1, ...]
 * A leaf has no child legs; the root's parent leg has dimension 1.
 *
 * Element types (enum cbc_dtype): float32, float64, complex64, complex128 (complex
 * numbers are interleaved (re, im) pairs).  The library computes in float64 or
 * complex128 storage; inputs of lower precision are widened on device at creation.
 *
 * Streams: every call is stream ordered on the cudaStream_t given at ttn_create of the
 * state (NULL = legacy default stream).  Device errors detected inside kernels are kept
 * in a status word and reported by the next call that synchronises (cbc_apply,
 * ttn_get_node, ttn_get_info).
 *
 * Device memory: stream-ordered allocations (networks, per-call workspaces) come from a
 * memory pool the library creates for itself on each device, which keeps freed memory
 * for reuse; the device's default memory pool is neither used nor reconfigured.
 *
 * Status: every function returns 0 (CBC_OK) or a positive cbc_status code; a message
 * for the calling thread is available from cbc_last_error().  No entry point aborts,
 * traps or leaves the process in an undefined state on bad input.
 */
#ifndef CBC_H_
#define CBC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cbc_ttn_s* ttn_t;   /* a TTNS / MPS held in device memory          */
typedef struct cbc_ttno_s* ttno_t; /* a TTNO / MPO held in device memory          */

enum cbc_status {
  CBC_OK = 0,
  CBC_ERR_INVALID_ARG = 1,        /* NULL pointer, bad dims, bad dtype, bad tree    */
  CBC_ERR_TOPOLOGY_MISMATCH = 2,  /* state and operator trees or phys dims differ   */
  CBC_ERR_OOM = 3,                /* device allocation failed                       */
  CBC_ERR_NOT_POSITIVE_DEFINITE = 4, /* Cholesky pivot <= 0 in CholeskyQR          */
  CBC_ERR_NUMERICAL = 5,          /* NaN / Inf met inside a kernel                  */
  CBC_ERR_TIMEOUT = 6,            /* a bounded device-side wait ran out             */
  CBC_ERR_CUDA = 7,               /* a CUDA runtime call failed                     */
  CBC_ERR_UNSUPPORTED = 8         /* valid request this build does not implement    */
};

enum cbc_dtype { CBC_F32 = 0, CBC_F64 = 1, CBC_C64 = 2, CBC_C128 = 3 };

/* Arithmetic of cbc_apply.
 * CBC_PREC_FP64 : every contraction, Gram matrix, eigensolve, Cholesky and triangular
 *                 solve in FP64 (the plain baseline).
 * CBC_PREC_MIXED: the dense contractions and Gram products run on the tensor cores
 *                 (tcgen05) with bf16 operand slices and FP32 partial sums that are
 *                 combined in FP64; the eigensolve, Cholesky and triangular solves stay
 *                 FP64.                                                             */
enum cbc_prec { CBC_PREC_FP64 = 0, CBC_PREC_MIXED = 1 };

typedef struct cbc_options {
  int precision;     /* enum cbc_prec; default CBC_PREC_FP64                         */
  int slices_fwd;    /* mixed: bf16 slices per operand in the first sweep(s) (0 = 5) */
  int slices_bwd;    /* mixed: bf16 slices per operand in the last sweep (0 = 4)     */
  int max_group;     /* cbc_apply_batched: most instances per lockstep group (0 = 32);
                        larger groups fill more SMs per launch and hold more memory    */
  double eps_rank;   /* singular values s_j <= eps_rank * s_0 are dropped (<= 0: the
                        default, 1e-12 for CBC_PREC_FP64 as in the FP64 reference, 1e-9
                        for CBC_PREC_MIXED, whose products resolve s only to ~3e-11 s_0) */
  double reserved_d[3];
} cbc_options;

/* Create a TTNS from node tensors.
 *   n_nodes   >= 1
 *   parent    [n_nodes] host array, -1 at the root, must describe one tree
 *   phys_dim  [n_nodes] host array, >= 1
 *   bond_dim  [n_nodes] host array, >= 1 (entry of the root ignored)
 *   dtype     enum cbc_dtype of node_data
 *   node_data [n_nodes] host array of pointers, each to one node tensor in the leg order
 *             above; host memory if data_on_device == 0, device memory otherwise.
 *             Tensors are copied: the caller keeps ownership and may free them after
 *             the call returns (it synchronises the stream when data is on the host).
 *   cuda_stream  cudaStream_t used by this handle and by cbc_apply on it (may be NULL)
 *   out       receives the new handle (owned by the caller, free with ttn_destroy)
 * Errors: CBC_ERR_INVALID_ARG, CBC_ERR_OOM, CBC_ERR_CUDA.                           */
int ttn_create(int n_nodes, const int32_t* parent, const int64_t* phys_dim,
               const int64_t* bond_dim, int dtype, const void* const* node_data,
               int data_on_device, void* cuda_stream, ttn_t* out);

/* Create a TTNO; same arguments as ttn_create with the operator leg order.  bond_dim
 * are the operator bonds (independent of the state's).                              */
int ttno_create(int n_nodes, const int32_t* parent, const int64_t* phys_dim,
                const int64_t* bond_dim, int dtype, const void* const* node_data,
                int data_on_device, void* cuda_stream, ttno_t* out);

/* Apply op to state and compress (Sec. III A for chains, Sec. III B for trees).
 *   max_bond  > 0: cap on every output bond; <= 0: no cap
 *   tol       > 0: keep the smallest rank whose discarded relative weight per cut
 *             sum_{j>=k} s_j^2 <= tol^2 sum_j s_j^2 (Sec. V adaptive bond); <= 0: off
 *   opt       NULL for defaults
 *   out       receives a new TTNS handle on the state's stream: non-root nodes are
 *             isometries toward the root (the Q^[i] of Eqs. (tt_cbc_qr_decomp),
 *             (cbc_tree_qr)); the root holds S^[root] divided by exp(log_norm)
 *             (ttn_get_info), so |psi'> = exp(log_norm) * network.
 * Truncation: the candidate directions of each compression come from the Gram matrix
 * and an eigensolver; the rank rule runs on weights measured on the factor itself
 * (||u_j^H M||^2 and, with tol > 0, the exact weight outside the candidates), and
 * directions the rule keeps below the Gram's resolution (weight < 1e-10 of the largest
 * in FP64, 1e-8 in the mixed path) are recomputed from the Gram of the residual.
 * The call is stream ordered; it synchronises the stream once per compressed bond to
 * read the weights back.  State and op are not modified.
 * Errors: CBC_ERR_INVALID_ARG, CBC_ERR_TOPOLOGY_MISMATCH, CBC_ERR_OOM,
 * CBC_ERR_NOT_POSITIVE_DEFINITE, CBC_ERR_NUMERICAL, CBC_ERR_TIMEOUT, CBC_ERR_CUDA,
 * CBC_ERR_UNSUPPORTED.  On error *out is left NULL and nothing leaks.               */
int cbc_apply(ttn_t state, ttno_t op, int64_t max_bond, double tol,
              const cbc_options* opt, ttn_t* out);

/* Apply n operators to n states (independent instances of any sizes and topologies)
 * and compress each; the results equal n calls of cbc_apply.  Tensor-train instances
 * with identical shapes (sites, physical and bond dimensions, real/complex), max_bond
 * and tol form groups of up to opt->max_group (default 32) that run in lockstep: every step of Sec. III A is one
 * launch for the whole group, on the stream of the group's first state (the group waits
 * for the other members' streams first and has finished when the call returns).  A
 * group whose members choose different ranks at some cut is rerun member by member.
 * Groups and the remaining instances are driven by up to `workers` host threads (<= 0:
 * min(#tasks, 16)) so their latency-bound steps overlap on the GPU; a lone instance j
 * runs on the stream of states[j], so give every state its own stream.
 *   max_bond, tol  [n] host arrays (per instance), or NULL for 0 (no cap / no tolerance)
 *   opt            shared by all instances (NULL for defaults)
 *   outs           [n] host array, receives the output handles (NULL where failed)
 * Returns the first failing status in instance order (CBC_OK if all succeeded); the
 * other instances still complete.                                                   */
int cbc_apply_batched(int n, const ttn_t* states, const ttno_t* ops, const int64_t* max_bond,
                      const double* tol, const cbc_options* opt, int workers, ttn_t* outs);

/* Zip-Up (Sec. III C): a comparison method that applies op
 * to state and compresses in a single sweep over the sites, truncating each bond as soon
 * as the site is contracted, with only the already compressed part in view.  Tensor
 * trains only (parent[i] = i - 1).  The sweep runs from the last site to site 0: at site
 * i the carried tensor (bond to site i+1 already compressed) is contracted with T^[i]
 * and W^[i] into Z[(alpha_{i-1} beta_{i-1}), (sigma'_i chi_i)]; the new tensor is an
 * orthonormal row basis of Z's dominant right singular subspace (rank rule of cbc_apply
 * on Z's singular values, max_bond and tol as there) and the carry is Z projected onto
 * it.  The state is used as given (no canonical form first).  Output layout, ownership,
 * precision options, stream use and errors as cbc_apply; CBC_ERR_UNSUPPORTED for a tree.
 * ttn_get_info's discarded weights are those of Z at each edge.                      */
int zipup_apply(ttn_t state, ttno_t op, int64_t max_bond, double tol,
                const cbc_options* opt, ttn_t* out);

/* The direct method (Sec. III C): a comparison method that
 * contracts op and state into one MPS (bond alpha_i beta_i on every edge) and compresses it
 * as a separate step.  Tensor trains only.  A QR sweep from site 0 makes sites 0 .. L-2
 * left-orthonormal (shifted CholeskyQR3 on the GPU), then a sweep from the last site to
 * site 0 truncates every edge by the rank rule of cbc_apply (max_bond, tol) on the Schmidt
 * values of the current state and keeps an orthonormal basis of the dominant right
 * singular vectors.  The product MPS holds d_i (alpha beta)^2 elements per site, so this
 * method needs far more memory than CBC.  Output layout, ownership, options, stream use
 * and errors as cbc_apply; CBC_ERR_UNSUPPORTED for a tree; ttn_get_info's discarded
 * weights are those of the truncating sweep.                                        */
int direct_apply(ttn_t state, ttno_t op, int64_t max_bond, double tol,
                 const cbc_options* opt, ttn_t* out);

/* Successive randomised compression, SRC (Sec. III C): a comparison method whose first
 * sweep contracts the network with one random matrix per site (d_i x s, joined across
 * the sites by the Khatri-Rao product: column j of every site's matrix belongs to the
 * same sketch vector) instead of compressing by an SVD; the second sweep is CBC's
 * (Eqs. (right_sweep_init_contr) .. (tt_cbc_final_contraction)) with the sketch in place
 * of the environments.  On the edge (i-1, i) the LQ takes the first
 * r = min(s, prod_{k<i} d_k, alpha_{i-1} beta_{i-1}) sketch rows (the generic rank of the
 * sketched block); when r is at least d_i chi_i the new tensor is the identity.  The
 * output bonds are therefore at most s; there is no tolerance rule.  Tensor trains only.
 *   sketch_size      s >= 1
 *   omega            [n_nodes] host array of pointers; omega[i] (i < n_nodes - 1) is the
 *                    d_i x s row-major random matrix of site i (the last site's entry is
 *                    not read and may be NULL), host or device memory per
 *                    omega_on_device; the caller draws them (e.g. standard Gaussian)
 *   omega_dtype      CBC_F32/CBC_F64 for real networks, CBC_C64/CBC_C128 for complex ones
 * The matrices are copied (FP64 storage) before the sweeps and freed on return; the call
 * synchronises the network's stream.  Output layout, ownership, options, errors as
 * cbc_apply (CBC_ERR_NOT_POSITIVE_DEFINITE when a sketched block is rank deficient, as for
 * a degenerate operator); CBC_ERR_INVALID_ARG for a bad sketch argument.             */
int src_apply(ttn_t state, ttno_t op, int64_t sketch_size, const void* const* omega,
              int omega_dtype, int omega_on_device, const cbc_options* opt, ttn_t* out);

/* The truncation rank rule of cbc_apply (Sec. III A compression to a bond cap, Sec. V
 * adaptive tolerance), on the host with no GPU work, for callers that want to predict or
 * check the bonds a compression chooses.
 *   n              number of candidate directions (>= 1)
 *   w              [n] host, their weights w_j = s_j^2 in descending order
 *   beyond         weight outside the candidates (0 when they span everything)
 *   max_bond, tol  as for cbc_apply
 *   floor_rel      rank floor: directions with s_j <= floor_rel * s_0 are dropped
 *   k_out          receives the kept rank: the prefix with w_j > floor_rel^2 w_0, then the
 *                  smallest k with sum_{j>=k} w_j + beyond <= tol^2 (sum_j w_j + beyond) when
 *                  tol > 0, then at most max_bond when max_bond > 0, at least 1
 *   discarded_out  NULL or receives the relative discarded weight of that choice
 * Errors: CBC_ERR_INVALID_ARG for n < 1, NULL w or k_out, or a non-finite argument.   */
int cbc_rank_rule(int n, const double* w, double beyond, int64_t max_bond, double tol,
                  double floor_rel, int* k_out, double* discarded_out);

/* Information about a TTNS (synchronises its stream).
 *   n_nodes_out     may be NULL
 *   bond_dims_out   NULL or [n_nodes]: bond of each node to its parent (1 at the root)
 *   log_norm_out    NULL or scalar: the network is scaled by exp(*log_norm_out)
 *   discarded_weight_out  NULL or [n_nodes]: for a result of cbc_apply, the relative
 *                   weight sum_{j>=k} s_j^2 / sum_j s_j^2 that the compression of the
 *                   edge from node i to its parent dropped (Sec. III A truncation; on a
 *                   chain the forward sweep's cut, on a tree the sum of the step-1 and
 *                   step-2 compressions of that edge); 0 at the root and for networks
 *                   made by ttn_create                                               */
int ttn_get_info(ttn_t t, int32_t* n_nodes_out, int64_t* bond_dims_out,
                 double* log_norm_out, double* discarded_weight_out);

/* Copy one node tensor out (synchronises the stream).
 *   dst   host (dst_on_device == 0) or device pointer with room for the node tensor
 *         in the leg order above, element type `dtype` (CBC_F64 or CBC_C128 for a
 *         complex network; CBC_F64 for a real one; lower precisions are rounded).   */
int ttn_get_node(ttn_t t, int node, void* dst, int dst_on_device, int dtype);

/* Copy every node tensor out at once (one synchronisation of the stream): node 0, then
 * node 1, ..., each in the leg order above, back to back without padding.
 *   dst   host (dst_on_device == 0) or device pointer with room for the sum over nodes
 *         of the node sizes (ttn_get_info gives the bonds), element type `dtype` as for
 *         ttn_get_node.
 * Errors: CBC_ERR_INVALID_ARG (NULL handle or pointer, dtype), CBC_ERR_CUDA.        */
int ttn_get_network(ttn_t t, void* dst, int dst_on_device, int dtype);

int ttn_destroy(ttn_t t);   /* NULL is a no-op */
int ttno_destroy(ttno_t t); /* NULL is a no-op */

/* Dense product used by every contraction of the sweeps, exposed as a building block
 * (and for kernel-level tests): C = op(A) op(B) with row-major DEVICE matrices of
 * dtype CBC_F64 or CBC_C128.  op(X) = X, X^T (trans), conj(X) (conj) or X^H (both).
 *   precision  CBC_PREC_FP64: FP64 SIMT; CBC_PREC_MIXED: tensor cores with `slices`
 *              bf16 slices per operand (2..5; 0 = 4), exact FP32 partial sums, FP64
 *              result (see cbc_apply)
 *   M, N, K    op(A) is M x K, op(B) is K x N, C is M x N (ldc >= N), K >= 1
 *   lda, ldb   leading dimensions of A and B as stored
 * Stream ordered on `stream`; allocates its workspace stream-ordered on it.
 * Errors: CBC_ERR_INVALID_ARG, CBC_ERR_OOM, CBC_ERR_CUDA.                           */
int cbc_gemm(int precision, int slices, int dtype, int M, int N, int K, const void* A,
             int64_t lda, int transA, int conjA, const void* B, int64_t ldb, int transB,
             int conjB, void* C, int64_t ldc, void* stream);

/* Truncation eigensolver, exposed as a building block (and for kernel-level tests).
 * The compression of Sec. III A keeps the dominant singular subspace of M; the sweeps
 * reach it through the Hermitian Gram matrix K = M M^H and this solver (Householder
 * reduction to tridiagonal form, Sturm multisection, inverse iteration, back
 * transformation).
 *   dtype    CBC_F64 or CBC_C128
 *   m, kmax  A is m x m Hermitian; the eigenvectors of the kmax largest eigenvalues
 *   nb       matrices in the batch, back to back (A: m*m apart, lam_out: m, U_out: m*kmax)
 *   A        DEVICE, row-major, overwritten
 *   lam_out  DEVICE, m doubles per matrix, descending: the first kmax are FP64 Rayleigh
 *            quotients of the computed vectors, the rest single-precision estimates
 *   U_out    DEVICE, m x kmax row-major per matrix, column j = eigenvector j
 *   mixed    nonzero: the mixed path's double-float reduction (used for batches, nb > 1)
 * Allocates its workspace stream-ordered on `stream` and synchronises it.
 * Errors: CBC_ERR_INVALID_ARG, CBC_ERR_OOM, CBC_ERR_TIMEOUT, CBC_ERR_CUDA.            */
int cbc_heev(int dtype, int m, int kmax, int nb, void* A, double* lam_out, void* U_out,
             int mixed, void* stream);

/* CholeskyQR2 of the backward sweep, exposed as a building block: the LQ of S on its row
 * leg (Eq. (tt_cbc_qr_decomp); Eq. (cbc_tree_qr) on trees) by G = S S^H, G = C C^H,
 * S <- C^{-1} S, twice, in FP64.
 *   S      DEVICE, m x n row-major with 1 <= m <= n, nb matrices m*n apart; replaced by Q
 *          with orthonormal rows spanning the row space of S
 * Synchronises the stream.  Errors: CBC_ERR_INVALID_ARG, CBC_ERR_OOM,
 * CBC_ERR_NOT_POSITIVE_DEFINITE (S rank deficient), CBC_ERR_TIMEOUT, CBC_ERR_CUDA.   */
int cbc_cholqr2(int dtype, int m, int n, int nb, void* S, void* stream);

/* Self-tests of device primitives the kernels rely on (no counterpart in the paper).
 * cbc_selftest_math: for n DEVICE doubles x, writes to the DEVICE array out[4 n]
 *   out[4i] = the library's Newton reciprocal of x_i (used where long chains of FP64
 *   divisions would dominate), out[4i+1] = 1.0 / x_i computed by CUDA, out[4i+2] = the
 *   library's Newton reciprocal square root (0 for x_i <= 0), out[4i+3] = CUDA's rsqrt.
 * cbc_selftest_wait: runs the library's bounded device-side wait on a word that nothing
 *   writes, with a limit of limit_cycles SM clock cycles; *returned_out = 1 when the
 *   kernel gave up and returned.  Returns CBC_ERR_TIMEOUT in that (expected) case: every
 *   wait of the library ends this way instead of hanging, and the context stays usable.
 * Both synchronise the stream.                                                       */
int cbc_selftest_math(const double* x_dev, double* out_dev, int64_t n, void* stream);
int cbc_selftest_wait(long long limit_cycles, int* returned_out, void* stream);

/* Launch statistics per kernel class, process wide, for benchmarks and profiling.
 * Launch counts are always kept.  With timing enabled, every group of launches of one
 * class is bracketed by CUDA events on the stream it runs on; cbc_stats_read then waits
 * for those events and sums their elapsed times.  flops are the algorithmic floating
 * point operations of the launches (8 per complex multiply-add, 2 per real one; a
 * Gram matrix counts only its Hermitian half).  Not thread safe across concurrent
 * cbc_apply calls.                                                                  */
enum cbc_kclass {
  CBC_K_GEMM_F64 = 0, /* FP64 SIMT contractions and Gram products                     */
  CBC_K_GEMM_TC = 1,  /* tcgen05 split-precision contractions and Gram products        */
  CBC_K_EIG = 2,      /* truncation eigensolver after the tridiagonal reduction        */
  CBC_K_CHOLQR = 3,   /* Cholesky and triangular solves of CholeskyQR2                */
  CBC_K_AUX = 4,      /* normalisation, identity, operand slicing, conversions        */
  CBC_K_TC_ISSUED = 5, /* flops only: bf16 products issued on the tensor pipe by the
                          split-precision GEMMs (S(S+1)/2 slice products on the padded,
                          real-embedded shape); no launches or time of its own          */
  CBC_K_TRIDIAG = 6,   /* Householder reduction to tridiagonal form (first stage of the
                          truncation eigensolver; CBC_K_EIG holds the other stages)     */
  CBC_K_COUNT = 8
};
typedef struct cbc_stats {
  int64_t launches[CBC_K_COUNT];
  int64_t groups[CBC_K_COUNT];
  double ms[CBC_K_COUNT];
  double flops[CBC_K_COUNT];
} cbc_stats;
int cbc_stats_enable(int timing); /* 1: time launch groups with CUDA events, 0: off  */
int cbc_stats_reset(void);
int cbc_stats_read(cbc_stats* out); /* synchronises the recorded events              */

/* Tensor-train CBC that allocates no device memory.
 *
 * The paper has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc (or any allocator) at the point where they need the application, e.g.
 * code running under a framework that owns every byte of device memory through its
 * own pool, or a real-time host loop in which allocation is forbidden after start-up.
 * It runs the same sweeps and kernels as cbc_apply on a chain in precision FP64 (the
 * same rank rule, and the identity as the new tensor wherever S has at least as many
 * rows as columns), but every intermediate lives in one library-owned scratch array of
 * CBC_NOALLOC_SCRATCH_BYTES, a file-scope __device__ array that each GPU which loads
 * the library holds until the process exits.
 *
 *   L            number of sites (chain rooted at site 0, as in ttn_create)
 *   phys_dim     [L] host, physical dimensions
 *   state_bond   [L] host, MPS bond of site i to site i-1 (entry 0 ignored)
 *   op_bond      [L] host, MPO bond of site i to site i-1 (entry 0 ignored)
 *   dtype        CBC_F64 or CBC_C128 (the caller widens lower precisions)
 *   state_nodes  [L] host array of DEVICE pointers, canonical leg order of ttn_create
 *   op_nodes     [L] host array of DEVICE pointers, canonical leg order of ttno_create
 *   max_bond, tol  as for cbc_apply
 *   out_data     DEVICE buffer of out_capacity elements of `dtype`; node i of the result
 *                (canonical layout, bonds out_bonds) starts at element out_offsets[i]
 *   out_offsets  [L] host, filled;  out_bonds [L] host, filled (1 at site 0)
 *   log_norm     host, filled: the result is exp(*log_norm) times the network
 *   cuda_stream  stream for all work (may be NULL)
 * The call synchronises the stream once per compressed bond (it reads the chosen rank
 * back to the host) and returns after the stream has drained, on success and on error.
 * The first call on a device looks up the device address of the scratch array on that
 * device (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call shares the one array and keeps nothing in it that a later call relies on
 * (it clears what must start at zero), so calls that overlap on the GPU, from several
 * threads or streams, race: serialise them.
 * Errors: CBC_ERR_INVALID_ARG for a NULL argument, a dimension < 1, a dimension product
 * beyond 2^31 - 1, intermediates that do not fit the scratch array (checked before
 * anything is launched; the message names the size needed) or a result larger than
 * out_capacity (checked once the forward sweep has fixed the ranks, before the
 * backward sweep writes anything; the message names the size needed); otherwise the
 * statuses of cbc_apply.                                                            */
#define CBC_NOALLOC_SCRATCH_BYTES (32u << 20)
int cbc_apply_tt_noalloc(int L, const int64_t* phys_dim, const int64_t* state_bond,
                         const int64_t* op_bond, int dtype, const void* const* state_nodes,
                         const void* const* op_nodes, int64_t max_bond, double tol,
                         void* out_data, int64_t out_capacity, int64_t* out_offsets,
                         int64_t* out_bonds, double* log_norm, void* cuda_stream);

/* Message of the last failing call on this thread ("" if none). */
const char* cbc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CBC_H_ */
