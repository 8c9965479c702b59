/*
 * pairdiag.h -- C ABI of the GB300 (sm_103a) ground-state solver for the
 * general pairing Hamiltonian in the seniority-zero pair basis.
 *
 *   H = sum_i (2 e_i + G_ii) n_i + sum_{i != j} G_ij P_i^+ P_j          (Eq. 2)
 *
 * Omega orbits (1 <= Omega <= 62), N pairs (0 <= N <= Omega).  A basis state
 * is an Omega-bit word with N set bits, bit p = orbit p (Sec. 3.1); basis
 * index r (0-based) is the state's position in ascending integer order, i.e.
 * the paper's hash value minus one (Sec. 3.2).  All vectors exchanged through
 * this ABI are in that order.
 *
 * Conventions for every entry point:
 *   - return value: PD_OK (0) on success, a negative PD_E* code otherwise;
 *     pairdiag_last_error() gives a one-line description of the last failure
 *     on the calling thread.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory on the handle's device (for example torch tensors'
 *     data_ptr()).  Nothing is retained after a call returns except what the
 *     handle owns.
 *   - kernels run on the handle's stream (pairdiag_set_stream; default: the
 *     legacy default stream).  Entry points taking host buffers synchronise
 *     that stream before returning; the *_dev entry points are asynchronous
 *     unless stated.
 *   - inputs are copied at create time; the caller keeps ownership of every
 *     buffer it passes.  The handle owns its device memory (basis tables,
 *     Lanczos window) and frees it in pairdiag_destroy.
 *   - threads: a solver or network handle serves one call at a time;
 *     different handles, the batch and odd-mass calls (each with its own
 *     network, if any), the autotuner's table and the device-memory cache may
 *     be used from several threads at once.  pairdiag_multidot_noalloc shares
 *     one scratch array per device (see its entry).  pairdiag_last_error() is
 *     per thread.
 */
#ifndef PAIRDIAG_H
#define PAIRDIAG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status ---- */
#define PD_OK        0
#define PD_EINVAL   -1   /* bad argument: Omega/N out of range, G not symmetric, non-finite input */
#define PD_ENOMEM   -2   /* device memory exhausted (dimension x window too large) */
#define PD_ENOCONV  -3   /* tolerance not reached in max_restarts; best estimate still returned */
#define PD_ETIMEOUT -4   /* a bounded device-side wait expired */
#define PD_ECUDA    -5   /* a CUDA runtime error */
#define PD_ENOTSUP  -6   /* request outside what this build supports */

/* precision of the Lanczos vectors and of H*x */
#define PD_PREC_FP64  0  /* FP64 vectors, FP64 row accumulation */
#define PD_PREC_MIXED 1  /* FP32 vectors + FP32 row sums; FP64 dots, FP64 tridiagonal
                            solve and a final FP64 Rayleigh-quotient refinement */
#define PD_HX_FLOATFLOAT 2  /* pairdiag_hx_dev only: float x, double y, float-float rows */

/* start vector of the first Lanczos cycle */
#define PD_START_RANDOM 0  /* counter-based SplitMix64 uniform in [-1,1), seeded */
#define PD_START_FIRST  1  /* [1,0,...,0]^T, the paper's default (Sec. 3.4) */
#define PD_START_HF     2  /* unit vector on the state of lowest diagonal element */
#define PD_START_USER   3  /* caller-provided vector (pairdiag_set_start) */
#define PD_START_MLP    4  /* product vector exp(sum_{i in s} w_i) with w from the learned
                              network (pairdiag_set_mlp) or given (pairdiag_set_start_weights) */

typedef struct pairdiag pairdiag_t;   /* opaque; owned by the library */

typedef struct {
    int      window;        /* Lanczos vectors per cycle (the paper's Lanc_Limit, Sec. 4.1); default 20 */
    int      max_restarts;  /* restart cycles before PD_ENOCONV; default 500 */
    int      precision;     /* PD_PREC_FP64 or PD_PREC_MIXED; default PD_PREC_FP64 */
    int      start;         /* PD_START_*; default PD_START_RANDOM */
    uint64_t seed;          /* seed of PD_START_RANDOM; default 1 */
    int      mode;          /* 0 = restarted Lanczos (the paper's Mode = 0), 1 = one Krylov
                               space without restart (Mode = 1); default 0 */
    int      low_bits;      /* orbits handled inside one basis block (0 = automatic) */
    double   mixed_floor;   /* relative residual at which FP32 cycles hand over to FP64
                               refinement (PD_PREC_MIXED only); default 5e-6 */
    int      hx_variant;    /* H*x kernel: 0 = automatic (default: the autotuned schedule if
                               one was recorded, else 3, or 4 with 13 low orbits when fewer
                               than 3 in 10 orbits are occupied or fewer than 3 in 10 empty), 1 = neighbour
                               blocks staged one at a time, 2 = all neighbour blocks staged at
                               once, 3 = no staging, every target gathered from global memory
                               with O(1) hop tables, 4 = variant 3 with the gathers issued in
                               deep groups (far from half filling, where a thread has one row
                               and x is in DRAM), 5 = variant 3 compiled for 5 resident
                               CTAs per SM (fewer registers, more warps); 2-5 fall back to 1
                               when their shared memory does not fit.  A truncated handle (pairdiag_truncate) runs
                               variant 1 */
} pairdiag_options;

typedef struct {
    int64_t dim;            /* C(Omega, N) */
    int64_t nnz_offdiag;    /* C(Omega,N) * N * (Omega - N) off-diagonal elements (Sec. 5.3) */
    int     iterations;     /* H*x products inside Lanczos (all precisions) */
    int     hx_products;    /* every H*x product of the call (Lanczos + FP64 refinement) */
    int     iterations_fp32;/* of which with FP32 vectors */
    int     restarts;       /* restart cycles */
    int     converged;      /* 1 if |beta_1/alpha_1| <= tol was reached */
    double  rel_residual;   /* ||Hv - E v|| / |E| of the returned vector (FP64) */
    double  gap_estimate;   /* second minus lowest Ritz value of the last cycle */
    double  seconds;        /* wall time of the call */
} pairdiag_info;

/* Fill *opt with the defaults listed above. */
void pairdiag_default_options(pairdiag_options *opt);

/* One-line description of a status code / of the last failure on this thread. */
const char *pairdiag_strerror(int code);
const char *pairdiag_last_error(void);

/*
 * Create a solver for Omega orbits and N pairs (the paper's N_Orbit, N_Pairs,
 * SPE and P_F inputs, Sec. 4.1; Initialize(), App. B).
 *   e : host, [omega] single-particle energies e_i
 *   G : host, [omega*omega] row-major pairing strengths, G[i*omega+j] = V_ij;
 *       must be exactly symmetric (the paper requires a real symmetric P_F).
 *   opt: host, nullable (defaults).
 *   out: receives the handle.
 * Builds the block tables for the basis on the current CUDA device.
 * Errors: PD_EINVAL (omega outside 1..62, N outside 0..omega, non-finite or
 * asymmetric input), PD_ENOMEM, PD_ECUDA.
 */
int pairdiag_create(int omega, int n_pairs, const double *e, const double *G,
                    const pairdiag_options *opt, pairdiag_t **out);

/* Free every device and host resource of the handle (the paper's Destory()). */
void pairdiag_destroy(pairdiag_t *h);

/* Run the handle's kernels on this CUDA stream (cudaStream_t passed as void*). */
int pairdiag_set_stream(pairdiag_t *h, void *stream);

/* Dimension of the space the solver works in, C(Omega,N) (Eq. extcmn) or the
 * kept states of a truncation (pairdiag_truncate), and the off-diagonal
 * nonzeros of the matrix there (Sec. 5.3).  Every vector of the ABI has
 * pairdiag_dim elements. */
int64_t pairdiag_dim(const pairdiag_t *h);
int64_t pairdiag_nnz(const pairdiag_t *h);
/* C(Omega,N), whether or not the handle is truncated. */
int64_t pairdiag_full_dim(const pairdiag_t *h);
/* The handle's number of orbits Omega (Eq. 2): the length of every per-orbit
 * host array (pairdiag_set_start_weights, pairdiag_product_start_dev, the
 * occupation numbers).  Host only, no device work; -1 for a null handle. */
int pairdiag_omega(const pairdiag_t *h);

/*
 * Basis states with indices [first, first+count) (Sec. 3.1, Table 1), written
 * as uint64 words to out_dev (device, [count]).  Bit-exact.  Asynchronous.
 * The basis, the ranks and pairdiag_monopole always describe the full space
 * of C(Omega,N) states, also on a truncated handle.
 */
int pairdiag_basis_dev(const pairdiag_t *h, int64_t first, int64_t count, uint64_t *out_dev);

/* The whole basis into host memory out (host, [C(Omega,N)]).  Synchronous. */
int pairdiag_basis(const pairdiag_t *h, uint64_t *out);

/*
 * Index of each state (the hash of Sec. 3.2, 0-based): ranks_dev[i] = f(states_dev[i]) - 1.
 * states_dev: device [count] Omega-bit words with N set bits (other words give
 * UINT64_MAX).  Asynchronous.
 */
int pairdiag_rank_dev(const pairdiag_t *h, const uint64_t *states_dev, int64_t count,
                      uint64_t *ranks_dev);

/*
 * y = H x computed on the fly (Sec. 3.3, Eq. diagonal), device buffers of dim
 * elements in basis order.
 *   precision PD_PREC_FP64: x_dev, y_dev are double; FP64 row sums.
 *   precision PD_PREC_MIXED: x_dev, y_dev are float; FP32 row sums, G rounded to FP32.
 *   precision PD_HX_FLOATFLOAT: x_dev is float, y_dev is double; every
 *     coefficient is split into two FP32 parts, each product with an element
 *     of x is exact in its high part, and the row sums are float-float, so the
 *     rows are as accurate as FP64 sums of the FP32 x while the arithmetic
 *     runs on the FP32 pipes.  The mixed form's FP64 Rayleigh refinement takes
 *     this product.  PD_ENOTSUP on a truncated handle or where its shared
 *     memory does not fit.
 * x_dev and y_dev must not overlap.  Asynchronous.
 */
int pairdiag_hx_dev(pairdiag_t *h, int precision, const void *x_dev, void *y_dev);

/* y = H x in FP64 with host buffers x, y of dim doubles (copies included).  Synchronous. */
int pairdiag_hx(pairdiag_t *h, const double *x, double *y);

/*
 * Monopole_Min, Monopole_Max and Posit_Min (Sec. 4.3, App. B): extreme
 * diagonal elements and the lowest index attaining the minimum.  Synchronous.
 */
int pairdiag_monopole(pairdiag_t *h, double *dmin, double *dmax, int64_t *pos_min);

/*
 * Truncated model space (Sec. 3.5, the paper's Dimension_Limit).  When
 * C(Omega,N) exceeds dimension_limit, the handle keeps only the states of
 * lowest diagonal element: every diagonal element (Eq. "diagonal", summed
 * in FP64 over the occupied orbits in ascending order) falls into one of
 * `bins` equal bins between the smallest and the largest,
 *     bin = min(floor((D - min) / (max - min) * bins), bins - 1)   (FP64),
 * and every state whose bin is at most the lowest bin at which the running
 * count from the bottom reaches dimension_limit is kept (so at least
 * dimension_limit states; whole bins).  A hop to a dropped state contributes
 * nothing: H on the kept states is the principal submatrix.
 *   dimension_limit : >= 1 to truncate; 0 restores the full space
 *   bins            : 1 .. 2^40; 0 = the paper's 10^8
 *   kept_dim        : host, receives the new pairdiag_dim
 * There is no truncation when C(Omega,N) <= dimension_limit or when every
 * diagonal element is equal.  After the call every vector of the ABI
 * (pairdiag_hx*, the ground and lowest states, pairdiag_set_start,
 * pairdiag_occupations_dev) holds the kept states in basis order; a start
 * vector set earlier is forgotten; PD_START_HF starts from the kept index of
 * the lowest state.  pairdiag_product_fit is not supported on a truncated
 * handle (PD_ENOTSUP).  The handle keeps C(Omega,N) int32 kept indices in
 * device memory.  Synchronous.
 */
int pairdiag_truncate(pairdiag_t *h, int64_t dimension_limit, int64_t bins, int64_t *kept_dim);

/* The kept index of every state of a truncated handle: map_dev (device,
 * int32 [C(Omega,N)]) receives the position of state r among the kept states,
 * or -1 when it is dropped.  PD_EINVAL when no truncation is active.
 * Asynchronous. */
int pairdiag_kept_map_dev(const pairdiag_t *h, int32_t *map_dev);

/*
 * Start vector for PD_START_USER: host [dim] doubles (copied).  Synchronous.
 */
int pairdiag_set_start(pairdiag_t *h, const double *v);

/*
 * Lowest eigenpair by restarted Lanczos (Algorithm 2 with full
 * reorthogonalisation and restart, Sec. 3.4; the paper's Diag_Solver).
 * Stops when |beta_1/alpha_1| <= tol (Sec. 5.1): the residual norm of the
 * restart vector relative to its Rayleigh quotient.  PD_PREC_MIXED runs FP32
 * cycles down to opt.mixed_floor, then FP64 Rayleigh refinement and, if
 * needed, FP64 cycles.
 *   e0  : host, receives the ground-state energy (Energy_Ground)
 *   vec : host [dim] doubles, nullable: the normalised ground-state vector
 *   info: host, nullable
 * Returns PD_OK, or PD_ENOCONV with the best estimate filled in.  Synchronous.
 */
int pairdiag_ground_state(pairdiag_t *h, double tol, double *e0, double *vec,
                          pairdiag_info *info);

/* As pairdiag_ground_state, with the vector written to device memory
 * (vec_dev: double [dim], nullable).  Synchronous (returns after E0 is known). */
int pairdiag_ground_state_dev(pairdiag_t *h, double tol, double *e0, double *vec_dev,
                              pairdiag_info *info);

/*
 * The k lowest eigenpairs ("the first few states" that Sec. 3.4 says are
 * wanted), one after another: state j is the ground state of the operator
 * projected against the converged states 0..j-1 (locking): every H*x result
 * and every restart vector of its Lanczos run is orthogonalised against them.
 * Each state runs the handle's form (FP64, or mixed with FP64 refinement) to
 * tol as pairdiag_ground_state does.  State 0 starts from the handle's start
 * kind; state j > 0 from the counter-based random vector of seed opt.seed + j
 * (a fresh start for each state, so that a degenerate level yields one state
 * per copy).
 *   k        : 1..min(64, dim)
 *   energies : host [k], in the order found (ascending up to tol)
 *   vecs_dev : device, nullable, [k * dim] doubles: state j at vecs_dev + j*dim,
 *              normalised, orthogonal to the earlier states up to tol
 *   info     : host [k], nullable, one record per state
 * Later pairdiag_ground_state calls on the handle see the whole space again.
 * Returns PD_OK, PD_ENOCONV if a state missed tol (all outputs filled), or
 * another PD_E* code.  Synchronous.
 */
int pairdiag_lowest_states_dev(pairdiag_t *h, int k, double tol, double *energies, double *vecs_dev,
                               pairdiag_info *info);

/*
 * Orbit occupation numbers 2 <v|S+_i S-_i|v> (N_Occup, Sec. 4.3) of a
 * normalised FP64 vector v_dev (device, [dim]); occ: host [omega].  Synchronous.
 */
int pairdiag_occupations_dev(pairdiag_t *h, const double *v_dev, double *occ);

/* ------------------------------------------------ learned warm start ---- */
/*
 * The paper starts Lanczos from [1,0,...,0] (Sec. 3.4) and has no learned
 * component; this warm start is an addition of this library.  A network maps
 * per-orbit features of (e, G, N) to weights w_i; the start vector is
 * psi(s) = exp(sum_{i in s} w_i - max).  Network: 16 -> 128 -> 128 -> 128 -> 1,
 * SiLU, bfloat16 operands with FP32 accumulation on the tensor cores
 * (tcgen05.mma, accumulators in tensor memory), FP32 master weights, Adam.
 * The entry points that run the network return PD_ETIMEOUT if a product's
 * bounded wait for its tensor-core operations expired.
 * Parameters (pairdiag_mlp_num_params() floats) are packed as W1 [16x128],
 * b1 [128], W2 [128x128], b2, W3 [128x128], b3, w4 [128], b4 [1], row-major.
 */
typedef struct pairdiag_mlp pairdiag_mlp_t;

/* New network with seeded initial weights on the current device. */
int  pairdiag_mlp_create(uint64_t seed, pairdiag_mlp_t **out);
void pairdiag_mlp_destroy(pairdiag_mlp_t *m);
int  pairdiag_mlp_num_params(void);
/* Copy the FP32 parameters out / in (host [num_params]); set resets Adam. */
int  pairdiag_mlp_get_params(const pairdiag_mlp_t *m, float *out);
int  pairdiag_mlp_set_params(pairdiag_mlp_t *m, const float *in);
/* Per-orbit input features of a problem: X host [omega x 16] floats. */
int  pairdiag_mlp_features(int omega, int n_pairs, const double *e, const double *G, float *X);
/* Network outputs for `rows` feature rows (host X [rows x 16] -> out [rows]). */
int  pairdiag_mlp_forward(pairdiag_mlp_t *m, int rows, const float *X, float *out);
/* One forward and backward pass: mean squared error against target [rows] and
 * its gradient (host [num_params]).  Test hook of the training kernels. */
int  pairdiag_mlp_loss_grad(pairdiag_mlp_t *m, int rows, const float *X, const float *target,
                            double *loss, float *grad);
/* `steps` full-batch Adam steps on (X, target); loss_history host [steps], nullable. */
int  pairdiag_mlp_train(pairdiag_mlp_t *m, int rows, const float *X, const float *target, int steps,
                        double lr, double *loss_history);
/* Intermediates of the network's last forward (and backward) pass, for
 * checking each layer on its own (test hook; the paper has no network):
 * which = PD_MLP_*, rows = the rows of that pass.  Activations and backward
 * intermediates stored in bfloat16 are widened to float.  out: host [rows *
 * 128] floats (PD_MLP_OUT, PD_MLP_DOUT: [rows]).  Synchronous. */
#define PD_MLP_Z1   0    /* X W1 + b1, FP32 */
#define PD_MLP_A1   1    /* silu(Z1), bfloat16 */
#define PD_MLP_Z2   2
#define PD_MLP_A2   3
#define PD_MLP_Z3   4
#define PD_MLP_A3   5
#define PD_MLP_OUT  6    /* A3 w4 + b4, FP32 */
#define PD_MLP_DOUT 7    /* 2 (out - t) / rows, FP32 (after a loss/gradient pass) */
#define PD_MLP_DZ3  8    /* dout w4 silu'(Z3), bfloat16 */
#define PD_MLP_DA2  9    /* dZ3 W3^T, FP32 */
#define PD_MLP_DZ2  10   /* dA2 silu'(Z2), bfloat16 */
#define PD_MLP_DA1  11   /* dZ2 W2^T, FP32 */
#define PD_MLP_DZ1  12   /* dA1 silu'(Z1), bfloat16 */
int  pairdiag_mlp_buffer(const pairdiag_mlp_t *m, int which, int rows, float *out);
/* Use the network for PD_START_MLP (the handle keeps the pointer; nullptr clears). */
int  pairdiag_set_mlp(pairdiag_t *h, pairdiag_mlp_t *m);
/* Use fixed weights w (host [omega]) for PD_START_MLP when no network is set. */
int  pairdiag_set_start_weights(pairdiag_t *h, const double *w);
/* Training target: the per-orbit weights w (host [omega], mean zero) that
 * minimise sum_s v_s^2 (log|v_s| - sum_{i in s} w_i)^2 for a normalised FP64
 * vector v_dev (device [dim]).  Synchronous. */
int  pairdiag_product_fit(pairdiag_t *h, const double *v_dev, double *w);
/* The product vector exp(sum_{i in s} w_i - max) into v_dev (device [dim], FP64). */
int  pairdiag_product_start_dev(pairdiag_t *h, const double *w, double *v_dev);

/* ------------------------------------------------------------- batch ---- */

typedef struct {
    int    iterations;      /* Lanczos H*x products of this problem */
    int    converged;       /* 1 if its residual reached tol */
    int    stalled;         /* mixed form: FP32 cycles stopped at their rounding floor */
    double rel_residual;    /* relative residual of the returned energy's vector: FP64
                               ||Hv - Ev||/|E| after refinement (mixed), else |beta_1/alpha_1| */
    double latency_ms;      /* device clock from the start of the call's device work to the
                               moment this problem's returned energy was final (after the
                               FP64 refinement in the mixed form) */
} pairdiag_batch_result;

/*
 * Ground states of `count` independent pairing Hamiltonians (Eq. 2): the
 * mean-field use case of Sec. 1/6, where a pairing solve sits inside every
 * self-consistent iteration.  The problems are sorted by dimension and split
 * into up to four size classes (the smallest 50 %, then 30 %, 15 % and 5 %;
 * one class below 64 problems), each on its own stream, the smaller ones at a
 * higher stream priority, so that small problems are not held back by the
 * largest.  Within a class the problems run restarted Lanczos in lock step:
 * every kernel serves all of them in one launch and converged problems drop
 * out.  The restart cycles of a class are one CUDA graph whose conditional
 * WHILE node repeats the cycle until a device-side test finds no problem
 * running (or max_restarts is reached): the host does not synchronise between
 * cycles.  The mixed form synchronises once per class after the FP64
 * refinement, to start FP64 cycles for problems that need them.
 *   omega, n_pairs : host [count]
 *   e_all          : host, the e vectors of all problems concatenated (sum of omega)
 *   G_all          : host, the row-major G matrices concatenated (sum of omega^2);
 *                    each exactly symmetric
 *   tol            : |beta_1/alpha_1| (Sec. 5.1); the mixed form refines every
 *                    vector in FP64 and reports that residual instead; problems
 *                    whose refined residual misses tol continue in FP64 cycles from
 *                    the refined vector
 *   opt            : nullable; window, max_restarts, precision, seed, low_bits and
 *                    mixed_floor are used; start PD_START_RANDOM or PD_START_MLP, mode 0
 *   mlp            : the warm-start network for PD_START_MLP (else nullable); one
 *                    network pass serves the orbits of all problems
 *   e0, status     : host [count] outputs (PD_OK or PD_ENOCONV per problem)
 *   results        : host [count], nullable
 *   stream         : cudaStream_t as void* (nullptr = legacy default stream)
 * Device memory is allocated for the call and freed before it returns.
 * Returns PD_OK, PD_ENOCONV if any problem missed tol (all outputs filled), or
 * another PD_E* code.  Synchronous.
 */
int pairdiag_batch_ground_state(int count, const int *omega, const int *n_pairs, const double *e_all,
                                const double *G_all, double tol, const pairdiag_options *opt,
                                pairdiag_mlp_t *mlp, double *e0, int *status,
                                pairdiag_batch_result *results, void *stream);

/* ---------------------------------------------------------- odd mass ---- */
/*
 * Odd-mass ground state in the blocking approximation (Eq. 3; the paper's
 * half-integer N_Pairs with its Block argument, Sec. 4.2).  The unpaired
 * particle occupies orbit b and keeps every pair out of it, so the subspace
 * with b blocked is the seniority-zero space of n_pairs pairs on the other
 * omega-1 orbits, and
 *     E_b = e_b + E0(Eq. 2 with e and G restricted to the orbits i != b).
 * Subspaces of at most 2^17 states with block = -1 and a PD_START_RANDOM or
 * PD_START_MLP start are solved together by the batched solver
 * (pairdiag_batch_ground_state) and, when vec or occ is wanted, the winning
 * subspace once more as a handle for its vector and occupations (e0 and
 * energies stay those of the batched solve; info describes the second solve).
 * Otherwise each subspace is a handle of this library on the restricted
 * (e, G); with block = -1 up to three library-internal host threads solve
 * them at once, each on a stream of its own.  Everything runs on the device
 * current when the call is made.
 *   omega, n_pairs : omega in 2..62, n_pairs in 0..omega-1 (2*n_pairs+1 particles)
 *   e, G           : host, as in pairdiag_create (G exactly symmetric)
 *   block          : -1 = every b, the lowest E_b is returned (the paper's Block = 0);
 *                    b in 0..omega-1 = that subspace alone (the paper's Block = b+1)
 *   tol, opt       : as in pairdiag_ground_state / pairdiag_create; tol is relative to
 *                    the pair part's Rayleigh quotient, without the constant e_b.
 *                    PD_START_USER is rejected (there is one vector per subspace)
 *   mlp            : the warm-start network for PD_START_MLP (else nullable)
 *   e0             : host, receives E_b of the returned subspace
 *   block_out      : host, nullable, receives its b
 *   energies       : host [omega], nullable, E_b of every solved b, NaN for the others
 *   occ            : host [omega], nullable, N_Occup of the returned state (Sec. 4.3):
 *                    2<S+_i S-_i> on the paired orbits, 1 on the blocked orbit
 *   vec            : host [C(omega-1, n_pairs)] doubles, nullable: the returned pair
 *                    vector, normalised, in the basis of the omega-1 unblocked orbits
 *                    renumbered 0..omega-2 in their original order
 *   info           : host, nullable: the returned subspace's solve; seconds covers
 *                    the whole call
 * Returns PD_OK, PD_ENOCONV if a solved subspace missed tol (all outputs
 * filled with the best estimates), or another PD_E* code.  Synchronous.
 */
int pairdiag_odd_ground_state(int omega, int n_pairs, const double *e, const double *G, int block,
                              double tol, const pairdiag_options *opt, pairdiag_mlp_t *mlp,
                              double *e0, int *block_out, double *energies, double *occ,
                              double *vec, pairdiag_info *info);

/* --------------------------------------------------------- autotuner ---- */
/*
 * H*x schedule autotuner (an addition of this library; the paper has a single
 * CPU code path).  For one problem and precision it times the H*x kernel for
 * every block split L = low_bits in [min(omega,8), min(omega,13)] and the five
 * kernel variants (median of `reps` launches on a random vector, CUDA events)
 * and records the fastest (low_bits, hx_variant) for (omega, n_pairs,
 * precision) in a process-wide table.  pairdiag_create and the batched solver
 * use a recorded schedule when opt.low_bits and opt.hx_variant are 0.
 *   best: host, receives the fastest; all: host [*n_all] (nullable), receives every
 *   timed candidate, *n_all = capacity on entry, count on return.  Synchronous;
 *   allocates and frees its own vectors and handles.
 */
typedef struct {
    int    low_bits;
    int    hx_variant;
    double ms;              /* median H*x duration */
} pairdiag_tune_entry;

int pairdiag_autotune(int omega, int n_pairs, const double *e, const double *G, int precision, int reps,
                      pairdiag_tune_entry *best, pairdiag_tune_entry *all, int *n_all);
/* Record (low_bits > 0) or clear (low_bits == 0) a schedule / read it (0, 0 if none). */
int pairdiag_tune_set(int omega, int n_pairs, int precision, int low_bits, int hx_variant);
int pairdiag_tune_get(int omega, int n_pairs, int precision, int *low_bits, int *hx_variant);

/* ------------------------------------------------------ device memory ---- */

/*
 * The library keeps the device blocks of destroyed handles (and of finished
 * batch calls) in a process-wide cache, per device and rounded size, and hands
 * them to the next handle that needs the same sizes: a loop of create / solve /
 * destroy then allocates once.  The paper has no counterpart (its Fortran
 * allocates host arrays).  When cudaMalloc runs out of memory the cache is
 * emptied once and the allocation retried.  Other allocators of the process
 * (PyTorch's caching allocator, for instance) cannot reclaim the cached
 * blocks themselves: release them before large allocations elsewhere.
 * pairdiag_release_cache returns every cached block to the driver (cudaFree);
 * released_bytes (nullable, host) receives their total size.  Blocks still
 * owned by live handles are not touched.  Thread-safe; always PD_OK.
 */
int pairdiag_release_cache(size_t *released_bytes);

/* ------------------------------------------------------- diagnostics ---- */

/* Number of CUDA kernels this library has launched since it was loaded (all
 * handles, all threads).  Host-side counter; never synchronises. */
int64_t pairdiag_kernel_launches(void);

/*
 * Kernel timing of the handle's H*x launches: while enabled (on != 0), every
 * H*x launch of the handle is bracketed by CUDA events on the handle's stream,
 * and so is the vector work of every Lanczos step that follows a product (the
 * fused step launch, or the recurrence/projection and update launches, with
 * the projection against locked states where there are any).
 * pairdiag_get_profile synchronises the stream, returns the number of timed
 * regions of the given kind and their summed duration in milliseconds, and
 * clears the records it returned (those of other kinds stay).  Kinds:
 * PD_PREC_FP64 or PD_PREC_MIXED (= FP32) H*x launches, a negative value for
 * both; 2 + PD_PREC_FP64 or 2 + PD_PREC_MIXED for the steps on FP64 or FP32
 * vectors.
 */
int pairdiag_set_profiling(pairdiag_t *h, int on);
int pairdiag_get_profile(pairdiag_t *h, int precision, int64_t *hx_launches, double *hx_ms);

/*
 * Form of the vector work of one Lanczos step after its product (Algorithm 2
 * with full reorthogonalisation, Sec. 3.4: the three-term recurrence, one
 * Gram-Schmidt pass against every vector of the window, the norm, the scaling
 * into the next basis vector).  on != 0 (default): one cooperative launch with
 * two grid-wide barriers, each CTA keeping its slice of the work vector in
 * shared memory where it fits; a barrier wait that gives up (after about a
 * second) makes the solve return PD_ETIMEOUT.  on == 0: three launches (two
 * streaming kernels whose sums are finished by their last CTA, and the
 * scaling).  Devices without cooperative launch always take the second form.
 * The results agree to rounding.  Applies from the next solve.
 */
int pairdiag_set_step_fusion(pairdiag_t *h, int on);

/*
 * Fused multiply-add throughput of the current device in the arithmetic of
 * one H*x nonzero (PD_PREC_FP64: FP64 FMA; PD_PREC_MIXED: FP32 FMA): a kernel of
 * independent FMA chains on every SM, timed with CUDA events on `stream` after
 * a warm-up launch (median of `reps` launches).  *tflops = 2 x FMAs / second
 * / 1e12.  The paper has no counterpart; it is the ALU roof of the FP64 H*x
 * product, which executes one FMA per nonzero.  Synchronous.
 */
int pairdiag_fma_peak(int precision, int reps, void *stream, double *tflops);

/* ------------------------------------------------ test hooks (device) ---- */

/*
 * Multi-dot with FP64 accumulation: out[j] = sum_i Q[j*ld + i] * p[i] for
 * j < m (m <= 64), n elements.  dtype 0 = double, 1 = float storage.
 * Q_dev, p_dev: device; out: host [m].  Synchronous.  (The reorthogonalisation
 * projections of Sec. 3.4.)
 */
int pairdiag_multidot(pairdiag_t *h, int dtype, const void *Q_dev, int64_t ld, int m,
                      const void *p_dev, int64_t n, double *out);

/*
 * Lowest eigenvalue (to FP64 accuracy), the second-lowest (to FP32 accuracy,
 * a gap estimate) and the lowest eigenvector of the symmetric tridiagonal
 * matrix with diagonal alpha[m] and off-diagonal beta[m-1] (the L matrix of
 * Algorithm 2; QR_Decompose in App. B), computed by the device solver.
 * alpha, beta: host; theta: host [2]; s: host [m].  m <= 64.  Synchronous.
 */
int pairdiag_tridiag_lowest(pairdiag_t *h, int m, const double *alpha, const double *beta,
                            double *theta, double *s);

/*
 * pairdiag_multidot_noalloc -- the multi-dot of pairdiag_multidot for callers
 * that cannot allocate device memory.  (The paper has no counterpart: this is
 * an interface addition of this library.)
 *
 * Some callers must not allocate: cudaMalloc and cudaFree can synchronise the
 * whole device, which a latency-critical host loop cannot afford, and some
 * host applications give a library no device memory beyond the buffers they
 * pass in.  This entry point needs no handle and calls no allocating routine:
 * its partial sums go to a fixed device array inside the library (524,288
 * bytes, held on every GPU that loads the library until the process exits).
 *
 *   out_dev[j] = sum_{i<n} Q_dev[j*ld + i] * p_dev[i],  j < m,  FP64 accumulation
 *   dtype : 0 = double storage, 1 = float storage (Q and p alike)
 *   Q_dev, p_dev, out_dev : device pointers; out_dev holds m doubles
 *   m     : 1..64 (larger m is rejected with PD_EINVAL: the fixed array holds
 *           partial sums for at most 64 vectors); 0 <= n <= ld
 *   stream: cudaStream_t as void* (nullptr = legacy default stream)
 * Asynchronous on `stream`.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) while that device is current; make
 * that first call before any stream capture begins.  All calls share the one
 * array and every call overwrites what it reads, so results never depend on an
 * earlier call -- but calls whose kernels overlap on the GPU (different streams
 * or threads without ordering between them) race on the array and must be
 * serialised by the caller.
 */
int pairdiag_multidot_noalloc(int dtype, const void *Q_dev, int64_t ld, int m, const void *p_dev,
                              int64_t n, double *out_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PAIRDIAG_H */
