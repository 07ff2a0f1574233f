/*
 * gcamps.h -- C ABI of libgcamps, a GB300 (sm_103a) implementation of the per-non-Clifford-gate
 * step of GCAMPS (Generalised Clifford Augmented Matrix Product States, arxiv 2511.06672).
 *
 * The state is psi = C |MPS> (Sec. 3): C is a Clifford kept as a mod-d stabilizer tableau
 * (Sec. 2.3), |MPS> a matrix product state (Sec. 2.4, Eq. mps).  Everything lives in device
 * memory owned by the handle; every step of a call runs in CUDA kernels of this library.
 *
 * Conventions (all calls):
 *   - d is 2 or 3 (Gaussian elimination over Z_d needs a field, Sec. 2.3.1; d > 3 is out of
 *     scope as in Sec. 3.1).  omega = exp(2 pi i/d), tau = exp(i pi/d).
 *   - A Weyl operator with phase is tau^r (x)_j X_j^{x_j} Z_j^{z_j}, r mod 2d (Sec. 2.3: Y = XZ
 *     for odd d, tau XZ for even d).
 *   - Qudit 0 is the most significant digit of a basis index: index = sum_j s_j d^{n-1-j}.
 *   - A Clifford on qudits (q0, q1) is given by the images of X_q0, Z_q0, X_q1, Z_q1 under
 *     conjugation U g U^dag: img[5k .. 5k+4] = (x_q0, z_q0, x_q1, z_q1, r) for generator k.
 *     One-qudit Clifford (q1 = -1): img[3k .. 3k+2] = (x, z, r), k = 0 (X), 1 (Z).
 *     The images must be symplectic and have order d (r even for odd d; for d = 2 each image
 *     Hermitian); otherwise the call returns GCAMPS_EINVAL and changes nothing.
 *
 * Ownership: input arrays are caller-owned host memory, read during the call only.  Output
 * arrays are caller-owned host memory written before the call returns.  A handle is used by
 * one host thread at a time and runs all its work on one CUDA stream (opts.cuda_stream, or a
 * stream the handle creates).
 *
 * Errors: every int-returning call returns 0 (GCAMPS_OK) or a GCAMPS_E* code; the message is
 * available from gcamps_last_error.  Calls that only enqueue device work (apply_*, disentangle,
 * run) are asynchronous: a device-side failure they cause (GCAMPS_ENOCONV, an iteration cap hit
 * inside a kernel, or GCAMPS_ECHI) is reported by the next call that synchronises
 * (gcamps_sync and every getter).  After EINVAL or ENOCONV the handle stays valid.
 */
#ifndef GCAMPS_H_INCLUDED
#define GCAMPS_H_INCLUDED

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GCAMPS_OK 0
#define GCAMPS_EINVAL 1  /* bad argument, non-symplectic images, unsupported d       */
#define GCAMPS_ENOMEM 2  /* device or host allocation failed                         */
#define GCAMPS_ECUDA 3   /* a CUDA runtime call failed                                */
#define GCAMPS_ENOCONV 4 /* a device iteration (the Jacobi SVD's sweeps) hit its cap   */
#define GCAMPS_ECHI 5    /* chi_max bound while discarding weight above strict_weight */
#define GCAMPS_ESIZE 6   /* a size beyond the fixed maximum of gcamps_score_theta_noalloc */
#define GCAMPS_ESNAP 7   /* the adjoint snapshot arena (opts.snapshot_entries) is full      */

typedef struct gcamps gcamps_t;

/* Run-time options (defaults from gcamps_default_opts). */
typedef struct {
  double cutoff;       /* keep singular values s_i > cutoff * s_0 (Sec. 2.4; default 1e-12)   */
  int max_sweeps;      /* disentangling sweeps per call (default 8)                           */
  int score_kind;      /* disentangler score (Sec. 3; Sec. 4 "bond-dimension criterion"):      */
                       /* 0 = von Neumann entropy of the normalised Schmidt spectrum;         */
                       /* 1 = Renyi-2 entropy -ln sum p^2;                                     */
                       /* 2 = number of Schmidt weights p > max(1e-12, 4 cutoff^2), ties       */
                       /*     broken by the von Neumann entropy                               */
  int precision;       /* 0 = FP64 contractions and scores; 1 = precision form: the class scores'  */
                       /* contractions (Q theta and its Gram) in FP32, tensor cores (tcgen05 TF32, */
                       /* three-term split) at CTA-level sizes, the Gram promoted to FP64 for the  */
                       /* FP64 reduction, eigenvalues and score; SVD splits FP64; tie_tol at least */
                       /* 1e-5 (the scores' FP32 resolution)                                      */
  double tie_tol;      /* accept Q only if S(Q) < S(I) - tie_tol; ties -> lowest index (1e-10) */
  void* cuda_stream;   /* cudaStream_t to run on, or NULL for a handle-owned stream            */
  /* The fields above are the contract's options, in its order; the ones below extend it.           */
  double strict_weight;/* if > 0: GCAMPS_ECHI when one truncation discards more than this      */
  int cluster_size;    /* CTAs (one thread-block cluster) per circuit: 1 to 16; 0 = 8            */
  int64_t snapshot_entries;   /* per circuit: complex entries of the arena that keeps the MPS  */
                              /* after every non-Clifford gate for gcamps_expect_gradient    */
                              /* (0 = no snapshots, no gradients; default 0)                 */
  int32_t snapshot_max_gates; /* per circuit: most non-Clifford gates kept (0 with the above) */
} gcamps_opts;

/* Per-circuit counters since creation (or gcamps_reset). */
typedef struct {
  int64_t t_gates;            /* non-Clifford gates applied                                 */
  int64_t clifford_gates;     /* Clifford gates applied to the tableau                      */
  int64_t bonds_visited;      /* disentangler bond visits                                   */
  int64_t candidates_scored;  /* (bond, class) entanglement scores evaluated                */
  int64_t accepted;           /* disentanglers applied                                      */
  int64_t sweeps;             /* disentangling sweeps                                       */
  int64_t vn_evaluations;     /* exact (FP64) von Neumann entropies computed; the other     */
                              /* classes were excluded by the Renyi-2 lower bound S2 <= S_vN */
                              /* or by their FP32 estimate's error bound                    */
  int64_t svd_calls;          /* truncating SVDs (one-sided Jacobi)                         */
  int64_t jacobi_sweeps;      /* Jacobi sweeps over all SVDs                                */
  int64_t jacobi_max_sweeps;  /* most sweeps one SVD needed                                 */
  int64_t qr_calls;           /* Householder QRs (canonical-form moves)                     */
  int32_t max_chi;            /* largest bond dimension seen after any truncation           */
  int32_t status;             /* sticky device status: 0 or a GCAMPS_E* code                */
  double discarded_weight;    /* sum of discarded s_i^2 over all truncations                */
  double scoring_flops;       /* algorithmic FP64 flops of exact class scoring (see below)  */
  double screen_flops;        /* algorithmic FP32 flops of the Renyi-2 screen (see below)   */
  double tensor_flops;        /* algorithmic flops of the Grams run on the tensor cores     */
                              /* (precision form: 8 m^2 K per m x m Gram of K columns)      */
  double algorithmic_flops;   /* the exhaustive search's flops: every class of every visit  */
                              /* with m > 1 scored exactly (the per-class FP64 count below), */
                              /* whether or not the bounds excluded it                      */
} gcamps_stats;
/* Per class at a bond with R = chi_l d rows and C = d chi_r columns (m = min(R, C),
 * M = max(R, C)): scoring_flops adds 8 d^2 R C (Q theta) + 4 m (m + 1) M (Hermitian Gram) +
 * (16/3) m^3 (Householder tridiagonalisation) per exact von Neumann evaluation (FP64; the
 * eigenvalue multisection is not counted); screen_flops adds 8 d^2 R C + 4 m (m + 1) M per class of
 * the FP32 Renyi-2 screen (every class of every bond with m > 1). */

/* One operation of a gate list (gcamps_run).  kind: */
#define GCAMPS_OP_CLIFFORD 1     /* q0, q1 (-1 for one qudit), img as for apply_clifford   */
#define GCAMPS_OP_NONCLIFFORD 2  /* q0 = site, phases[0..d-1]                             */
#define GCAMPS_OP_DISENTANGLE 3  /* disentangle the span of the last non-Clifford gate;    */
                                 /* q0 > 0: at most q0 sweeps (else opts.max_sweeps);      */
                                 /* q1 > 0: stop after q1 bond visits                      */
typedef struct {
  int32_t kind;
  int32_t q0, q1;
  int32_t img[20];
  int32_t pad;
  double phases[4];
} gcamps_op;

void gcamps_default_opts(gcamps_opts* o);

/* Number of two-qudit disentangler classes searched per bond: d^2 (d^2 + 1), i.e. 20 for d = 2
 * and 90 for d = 3 (Sec. 3).  Returns -1 for unsupported d. */
int gcamps_num_candidates(int d);

/* Images (img[20], layout as above) of the two-qudit Clifford  W(shift) U_S  where S is the
 * sp_index-th element (0-based) of Sp(4, F_d) in lexicographic order of its row-major entries
 * (column k = exponents of the image of generator k in coordinates (x_q0, z_q0, x_q1, z_q1)),
 * U_S maps each generator to the standard-phase Weyl operator of its column (phase tau^0 for
 * odd d, tau^{x_q0 z_q0 + x_q1 z_q1} for d = 2), and W(shift) = X^s0 Z^s1 (x) X^s2 Z^s3 acts after
 * it.  This is how the seeded benchmark circuits name their gates (the random two-qudit Cliffords of
 * the Sec. 4 benchmarks; Sp(4, F_d) as in Sec. 3.1).  EINVAL on bad arguments. */
int gcamps_sp4_images(int d, int64_t sp_index, const int32_t* shift, int32_t* img);

/* Host-only (no GPU needed): class k (0 <= k < gcamps_num_candidates(d)) of the disentangler set
 * (the 20 / 90 entangling classes of Sec. 3, built as in Sec. 3.1).
 * img[20]: generator images of its representative (class 0 = identity; the others are the
 * lexicographically smallest symplectic matrix of their class {(L_0 (+) L_1) S}, standard phases);
 * u: its d^2 x d^2 unitary, row-major, interleaved (re, im), 2 d^4 doubles (may be NULL). */
int gcamps_candidate(int d, int k, int32_t* img, double* u);

/* Named gates of Sec. 2.3 (phases in units of tau = exp(i pi / d), as everywhere in this ABI):
 *   H    H|i> = d^{-1/2} sum_j omega^{ij} |j>:           X -> Z,               Z -> X^{d-1}
 *   S    diag(omega^{j(j-1)/2}) (odd d), diag(1, i) (d = 2): X -> tau^{[d=2]} X Z, Z -> Z
 *   SUM  |i, j> -> |i, i + j> (q0 the control):          X_q0 -> X_q0 X_q1,    Z_q1 -> Z_q0^{d-1} Z_q1
 *                                                        (Z_q0 and X_q1 fixed)
 *   X    X|j> = |j + 1>:                                 Z -> omega^{-1} Z
 *   Z    Z|j> = omega^j |j>:                             X -> omega X               */
#define GCAMPS_GATE_H 1
#define GCAMPS_GATE_S 2
#define GCAMPS_GATE_SUM 3
#define GCAMPS_GATE_X 4
#define GCAMPS_GATE_Z 5
/* The same gate codes under the short names gcamps_apply_named is documented with. */
#define GCAMPS_H GCAMPS_GATE_H
#define GCAMPS_S GCAMPS_GATE_S
#define GCAMPS_SUM GCAMPS_GATE_SUM
#define GCAMPS_X GCAMPS_GATE_X
#define GCAMPS_Z GCAMPS_GATE_Z
/* Host-only (no GPU needed): generator images of a named gate, in the layout of
 * gcamps_apply_clifford (img: 6 ints for a one-qudit gate, 20 for SUM; the caller's buffer holds
 * at least that many).  *nq (may be NULL) receives the gate's qudit count.  EINVAL for an unknown
 * gate or unsupported d. */
int gcamps_named_images(int d, int gate, int32_t* img, int32_t* nq);

/* Create a simulator of `batch` independent circuits of n qudits (n >= 2), local dimension d,
 * bond dimension at most chi_max, all in |0...0> with C = I.  Device memory for the MPS is
 * reserved up front for bond dimension d * chi_max (the MPO growth of Sec. 2.4).
 * gcamps_create is gcamps_create_batch with batch = 1.  EINVAL (before any CUDA call) for bad
 * options, or when a matrix of the engine would exceed 2^31 - 1 entries: the two-site tensor after
 * the MPO, (d c) x (d c) with c = d min(chi_max, d^min(b, n-b)) the largest bond capacity. */
int gcamps_create(int n, int d, int chi_max, const gcamps_opts* o, gcamps_t** out);
/* `batch` independent circuits of the same n (Sec. 2.4 layout each, as above). */
int gcamps_create_batch(int batch, int n, int d, int chi_max, const gcamps_opts* o, gcamps_t** out);
/* gcamps_batch_create(count, n[], d, chi_max, o, out): the batched form's constructor, the same call as
 * gcamps_create_batch_uneven below (circuits with their own qudit counts, no counterpart in the paper). */
int gcamps_batch_create(int count, const int32_t* n, int d, int chi_max, const gcamps_opts* o, gcamps_t** out);
/* Batch of circuits with their own qudit counts n[c] (2 <= n[c] <= 128), for many independent
 * circuits of uneven size in one engine launch (gcamps_run with per-circuit op ranges).  Memory is
 * reserved per circuit for its own n[c]; calls that apply to every circuit (apply_*, disentangle)
 * require sites below the smallest n[c]; readouts use the circuit's own n[c].  No counterpart in the
 * paper (it runs one circuit at a time, Sec. 4.1.1). */
int gcamps_create_batch_uneven(int batch, const int32_t* n, int d, int chi_max, const gcamps_opts* o,
                               gcamps_t** out);
/* Waits for the handle's work, then frees it, its device memory and the stream it created (not a
 * caller's stream); NULL is ignored.  No counterpart in the paper. */
void gcamps_destroy(gcamps_t* h);
/* Qudits of circuit `circuit` (-1 for a bad handle or index).  No counterpart in the paper. */
int gcamps_num_qudits(gcamps_t* h, int circuit);
/* CTAs per circuit for the following launches: 1 up to the cluster size the handle was created with
 * (its per-CTA scratch is laid out for that many).  Synchronises the handle's stream.
 * Used to pick the fastest cluster size for a workload by measurement.  No counterpart in the paper
 * (a launch shape of this library).  EINVAL for other sizes. */
int gcamps_set_cluster_size(gcamps_t* h, int cluster_size);

/* Most sweeps one Jacobi SVD may take before the engine gives up with GCAMPS_ENOCONV (reported by the next
 * synchronising call; the circuit does no further MPS work until gcamps_reset).  Default 60.  Synchronises
 * the handle's stream; applies to the following launches.  No counterpart in the paper: an iteration cap of
 * this library, settable so that the failure path can be exercised.  EINVAL outside 1..1000. */
int gcamps_set_jacobi_cap(gcamps_t* h, int sweeps);

/* Where the exact FP64 class evaluations of a bond visit with m = min(chi_l d, d chi_r) <= 27 run: on one
 * warp each (many at once), or, when the visit's exact list has no more classes than the cluster has CTAs
 * and m >= min_m, on one CTA each.  The choice changes the summation order only (the same class is chosen
 * up to ties within rounding).  Default 10; 0 puts every such list on CTAs, a value above 27 keeps the
 * warps.  No counterpart in the paper: a launch-shape setting of this library (Sec. 3's class scores are
 * its subject).  Synchronises the handle's stream.  EINVAL if min_m < 0. */
int gcamps_set_exact_cta(gcamps_t* h, int min_m);

/* C <- G C for a one- or two-qudit Clifford G (Sec. 3, top loop of Fig. 3): the tableau rows
 * are conjugated (Table 1 generalised to any Clifford given by its images).  Applied to every
 * circuit of the handle. */
int gcamps_apply_clifford(gcamps_t* h, int q0, int q1, const int32_t* img);
/* gcamps_apply_clifford with the images of a named gate of Sec. 2.3 (gcamps_named_images): q1 = -1
 * for H, S, X, Z; for SUM q0 is the control and q1 the target.  EINVAL otherwise. */
int gcamps_apply_named(gcamps_t* h, int gate, int q0, int q1);

/* Diagonal non-Clifford gate diag(exp(i phases[j])), j = 0..d-1, on `site` (Sec. 2.3.2, Sec. 3):
 * P = C^dag Z_site C is read from the inverse tableau, the gate is expanded as
 * sum_m c_m Z^m and applied to the MPS as the d-term MPO sum_m c_m P^m over the support span
 * [f, l] of P, then [f, l] is recompressed (QR-equivalent sweep, then truncated SVD with
 * cutoff and chi_max).  Applied to every circuit of the handle. */
int gcamps_apply_nonclifford(gcamps_t* h, int site, const double* phases);

/* Disentangle the span of the last non-Clifford gate (Sec. 3): alternating sweeps over its
 * bonds; at each bond every class Q is scored by the entanglement entropy of Q theta, the best
 * one is applied if it lowers the entropy by more than tie_tol, and C <- C Q^dag.  st may be
 * NULL; if given it receives the counters of circuit 0 after the call (this synchronises).
 * Applied to every circuit of the handle. */
int gcamps_disentangle(gcamps_t* h, gcamps_stats* st);

/* Run a gate list on every circuit of the handle: both loops of Fig. 3 (Sec. 3) for every op in
 * order.  ops: host array; circuit c runs ops[begin[c] .. begin[c+1]) (begin has batch+1 entries;
 * NULL begin = all ops on every circuit).  One kernel launch for the whole list; asynchronous.
 * EINVAL (nothing enqueued) for a bad op or bad offsets. */
int gcamps_run(gcamps_t* h, const gcamps_op* ops, int nops, const int32_t* begin);
/* gcamps_run (Fig. 3, Sec. 3) with `ops_dev` and `begin_dev` already in device memory (no host-to-device copy; the ops
 * are not validated, so they must have passed through gcamps_run's checks before). */
int gcamps_run_device(gcamps_t* h, const gcamps_op* ops_dev, const int32_t* begin_dev);

/* <psi| W |psi> for W = (x)_j X_j^{x_j} Z_j^{z_j} (phase 1), as C^dag W C is a product of inverse
 * tableau rows and <MPS|.|MPS> a transfer-matrix contraction (Sec. 3).  O_sigma of Sec. 3 is
 * the real part.  x, z: n exponents each (0..d-1).  The handle's circuit 0 (the only one of a handle
 * from gcamps_create); gcamps_batch_expect_weyl takes the batch entry `circuit`.  Synchronising. */
int gcamps_expect_weyl(gcamps_t* h, const int32_t* x, const int32_t* z, double* re, double* im);
/* The same readout for batch entry `circuit` (Sec. 3). */
int gcamps_batch_expect_weyl(gcamps_t* h, int circuit, const int32_t* x, const int32_t* z, double* re, double* im);

/* Phase gradient of O = Re <psi| W |psi> = <psi| (W + W^dag)/2 |psi>, W = (x)_j X_j^{x_j} Z_j^{z_j},
 * with respect to the phases of every non-Clifford gate k applied since the last reset
 * (gate k = diag(exp(i phi_{k,j})), j = 0..d-1; Sec. 2.3.2 writes the T gate through R_Z(theta), so
 * theta-parametrised gates get d/dtheta by the chain rule).  Adjoint method through the MPO
 * applications (Sec. 3): the handle must be created with snapshots (opts.snapshot_entries,
 * snapshot_max_gates); the state after each gate's MPO is kept on the device, and the backward pass
 * runs in the forward run's own Clifford frames (undoing each disentangler, applying the inverse
 * gate's MPO), so it is exact when no truncation discards weight.  value: O; grad: d doubles per gate
 * (gate-major), at most cap_gates gates copied; *ngates: gates recorded.  Synchronising; uses a
 * workspace circuit slot, so one gradient at a time per handle.  GCAMPS_ESNAP if the arena was full;
 * GCAMPS_ECHI if chi_max made the backward pass discard weight (the backward state carries the
 * observable evolved back through the later gates and can need a larger bond dimension than the
 * forward state; the gradient would not be exact). */
int gcamps_expect_gradient(gcamps_t* h, int circuit, const int32_t* x, const int32_t* z, double* value,
                           double* grad, int32_t cap_gates, int32_t* ngates);

/* Dense psi = C|MPS> (Sec. 3; d^n amplitudes, d^n <= 2^20) up to one global phase (a Clifford given by its
 * images has no defined phase): C|y> = prod_j D_j^{y_j} C|0>, with C|0> the common +1
 * eigenvector of the stabilizer rows.  re/im: d^n doubles each. */
int gcamps_statevector(gcamps_t* h, int circuit, double* re, double* im);
/* One amplitude <s|C|MPS> (Sec. 3) with the same global-phase convention (d^n <= 2^20); digits: n values in
 * 0..d-1 (qudit 0 first).  Circuit 0 (gcamps_amplitude) or batch entry `circuit` (gcamps_batch_amplitude). */
int gcamps_amplitude(gcamps_t* h, const int32_t* digits, double* re, double* im);
/* The same readout for batch entry `circuit` (Sec. 3). */
int gcamps_batch_amplitude(gcamps_t* h, int circuit, const int32_t* digits, double* re, double* im);

/* Tableau of C (Sec. 2.2, Sec. 2.3): exps[2n][2n] (row-major; rows 0..n-1 = C Z_j C^dag, rows n..2n-1 = C X_j C^dag;
 * columns x_0..x_{n-1} | z_0..z_{n-1}) and phase[2n] (mod 2d, units of tau); either may be NULL.  Circuit 0
 * (gcamps_get_tableau) or batch entry `circuit` (gcamps_batch_get_tableau). */
int gcamps_get_tableau(gcamps_t* h, uint8_t* exps, uint8_t* phase);
/* The same readout for batch entry `circuit` (Sec. 2.2, Sec. 2.3). */
int gcamps_batch_get_tableau(gcamps_t* h, int circuit, uint8_t* exps, uint8_t* phase);
/* Inverse tableau: rows C^dag Z_j C (0..n-1) and C^dag X_j C (n..2n-1), same layout (the strings
 * that the Gaussian elimination of Sec. 2.3.1 produces, kept up to date instead). */
int gcamps_get_inverse_tableau(gcamps_t* h, int circuit, uint8_t* exps, uint8_t* phase);
/* Bond dimensions chi[0..n-2] of the MPS (Sec. 2.4; bond j joins qudits j and j+1).  Circuit 0
 * (gcamps_get_bond_dims) or batch entry `circuit` (gcamps_batch_get_bond_dims). */
int gcamps_get_bond_dims(gcamps_t* h, int32_t* chi);
/* The same readout for batch entry `circuit` (Sec. 2.4). */
int gcamps_batch_get_bond_dims(gcamps_t* h, int circuit, int32_t* chi);
/* Schmidt values of bond `bond` (Sec. 2.4; count <= chi of that bond), sorted descending. */
int gcamps_get_schmidt(gcamps_t* h, int circuit, int bond, double* s, int32_t* count);
/* Tensor of MPS site j (Sec. 2.4, Eq. mps): dims[0..2] = (chi_l, d, chi_r); if t is not NULL it receives the
 * chi_l d chi_r complex entries (interleaved re, im; row-major over (a, s, b)); cap = capacity of t
 * in complex entries (EINVAL if too small). */
int gcamps_get_site(gcamps_t* h, int circuit, int site, double* t, int64_t cap, int32_t* dims);
/* Weyl string P = C^dag Z_k C of the last non-Clifford gate (Sec. 2.3.1, Sec. 3): x[n], z[n], r. */
int gcamps_get_last_weyl(gcamps_t* h, int circuit, int32_t* x, int32_t* z, int32_t* r);
/* Counters of circuit `circuit` (gcamps_stats; no counterpart in the paper). */
int gcamps_get_stats(gcamps_t* h, int circuit, gcamps_stats* st);
/* Replay (the oracle's replay of Sec. 3 decisions, for comparing two runs of one circuit): from the next
 * launch, circuit `circuit` applies pairs[2k], pairs[2k+1] = (bond, class) at its k-th disentangler bond
 * visit instead of scoring the classes (gcamps_get_decisions gives such a list); each visit splits by SVD.
 * Visit k at another bond, or more visits than count, set GCAMPS_EINVAL in the circuit's status.  count = 0
 * turns replay off.  pairs: host memory, copied; bonds 0..n-2, classes 0..K-1 (EINVAL otherwise); count
 * <= 65536.  Synchronises the handle's stream; the first call allocates the replay buffers (ENOMEM). */
int gcamps_set_replay(gcamps_t* h, int circuit, const int32_t* pairs, int32_t count);

/* <M1|M2> of the MPS of circuit1 of h1 and circuit2 of h2 (Sec. 2.4; transfer matrices in FP64): with equal
 * tableaux (bit-exact, e.g. one run replaying the other's decisions) the two states C|M1>, C|M2> have
 * overlap <M1|M2> and fidelity |<M1|M2>|^2.  The handles need the same n, d and chi_max (EINVAL otherwise);
 * h2's stream is synchronised, the contraction runs on h1's stream in h1's scratch.  Synchronising. */
int gcamps_overlap(gcamps_t* h1, int circuit1, gcamps_t* h2, int circuit2, double* re, double* im);

/* Where the engine's time went for circuit `circuit` since creation (or gcamps_reset): no counterpart in
 * the paper, a measurement aid.  out receives min(cap, GCAMPS_PROF_WORDS) int64 words (*count, may be NULL,
 * receives GCAMPS_PROF_WORDS), all SM clock cycles (clock64) of the circuit's leader CTA, whose intervals
 * include its waits at the cluster's barriers, so the phases add up to the launch's time on that circuit:
 *   [0] Clifford tableau updates          [1] non-Clifford steps (MPO apply and recompression)
 *   [2] centre moves before a sweep       [3] forming theta at a bond visit
 *   [4] FP32 Renyi-2 screen of every class [5] FP32 von Neumann estimates (their bounds)
 *   [6] exact FP64 class evaluations       [7] the decision
 *   [8] applying the chosen class and folding it into the tableau
 *   [9] truncated SVD splits               [10] QR centre moves after a visit that applies nothing
 *   [12 + b] bond visits, [17 + b] their cycles, [22 + b] their exact evaluations, [27 + b] their FP32
 *   von Neumann estimates, for the visit size buckets b = 0..4 of m = min(chi_l d, d chi_r): m <= 9, <= 27,
 *   <= 54, <= 81, larger; [11] cycles and [32] count of the warp-level exact evaluations run by the leader
 *   CTA's first warp (the duration of one evaluation, free of the cluster's waits); [33 + 11 b + p] the
 *   cycles of phase p (0..10 as above) spent inside the visits of bucket b; [88 + 6 (5 g + b) + j] the
 *   leader CTA's own exact evaluations at warp level (g = 0, its first warp) or CTA level (g = 1) in bucket
 *   b: j = 0 their count, 1 their cycles, of which 2 forming theta' and its Gram, 3 the Householder
 *   reduction, 4 the eigenvalues, 5 the entropy; [160 + r] 1 + the SM id that cluster rank r (r < 16) ran
 *   on in the last gate-list launch (0: none); [191] internal (0 between launches). */
#define GCAMPS_PROF_WORDS 192
int gcamps_get_profile(gcamps_t* h, int circuit, int64_t* out, int32_t cap, int32_t* count);
/* Scores (Sec. 3) of the last disentangler bond visit of the circuit: s2[k] (Renyi-2 entropy of every class:
 * FP64 where evaluated[k] = 1, else the FP32 screening value, within 4 eta sqrt(m) + 4 eta of the exact
 * one with eta < 3 (d^3 + 6 d + max side) 2^-24), vn[k] (von Neumann entropy, valid where
 * evaluated[k] = 1 except for classes scored by Renyi-2 alone under score_kind 1, which read NaN;
 * the bounds excluded the others);
 * K = gcamps_num_candidates(d) entries each; any pointer may be NULL. */
int gcamps_get_last_scores(gcamps_t* h, int circuit, double* s2, double* vn, uint8_t* evaluated);
/* Two-site tensor theta scored at the last bond visit (Sec. 3): shape[0..1] = (chi_l, chi_r); theta receives the
 * chi_l d d chi_r complex entries (interleaved re, im) when that count is at most 729 (larger
 * tensors are not kept). */
int gcamps_get_last_theta(gcamps_t* h, int circuit, double* theta, int32_t* shape);
/* Disentangler decisions (Sec. 3, each folded as C~ = C Q^dag) of the circuit since the last reset: (bond, class index) per bond
 * visit, in visit order; class 0 = nothing applied.  *count receives the total number
 * recorded; at most cap pairs are copied. */
int gcamps_get_decisions(gcamps_t* h, int circuit, int32_t* pairs, int32_t cap, int32_t* count);

/* Disentangler scores of every class on a given two-site tensor (Sec. 3): theta is
 * chi_l x d x d x chi_r complex (interleaved re, im, row-major over (a, s, t, b)), on host memory.
 * s2[k] = Renyi-2 entropy and vn[k] = von Neumann entropy (natural log) of the Schmidt spectrum of
 * Q_k theta across (a, s) | (t, b), K = gcamps_num_candidates(d) entries each.  Runs the same device
 * code as gcamps_disentangle (every class evaluated here).  choice (may be NULL) receives the
 * class the disentangler would apply to this theta (0 = none) and how many exact entropies its
 * Renyi-2 pruning evaluated.  Synchronising. */
int gcamps_score_theta(gcamps_t* h, int chi_l, int chi_r, const double* theta, double* s2, double* vn,
                       int32_t* choice);

/* FP32 estimates of the von Neumann entropy (Sec. 3 score) of every class on a given two-site tensor, with
 * the error bound the disentangler prunes with: theta' = Q_k theta and its Gram in FP32, scaled to unit
 * trace, reduced to a tridiagonal by FP32 Householder reflections, eigenvalues by FP32 multisection;
 * |est[k] - S_vN(Q_k theta)| <= bound[k] (bound[k] = 1e300 where it carries no information: large Grams,
 * or a trace outside 1e-12 .. 1e12).  The bound is twice the Fannes-Audenaert bound of a trace distance
 * T = sqrt(m) (eta + u + 2 m^2 u (1 + eta)) + 9 m u (u = 2^-24; eta the FP32 Gram error of the screen;
 * 2 m^2 u |G|_F the backward error of the FP32 reduction).  theta as for gcamps_score_theta (host memory);
 * est, bound: K doubles each.  Synchronising. */
int gcamps_estimate_theta(gcamps_t* h, int chi_l, int chi_r, const double* theta, double* est, double* bound);

/* The class scores of gcamps_score_theta for callers that cannot allocate device memory: code
 * whose GPU memory belongs to another allocator (a framework's memory pool that has already
 * reserved the device, or a fixed per-process memory budget), and latency-critical loops that
 * cannot take the device-wide synchronisation cudaMalloc and cudaFree may cause.  The paper has no
 * counterpart of this call; it is a deployment variant of the disentangler scoring.
 *
 * It needs no handle and allocates nothing (no cudaMalloc, no cudaFree, no allocating library
 * routine).  Its working memory is one static device array of this library, 1,696,256 bytes, that
 * every GPU which loads the library holds until the process exits.  That array fixes the largest
 * tensor: chi_l d <= GCAMPS_NOALLOC_MAX_SIDE and d chi_r <= GCAMPS_NOALLOC_MAX_SIDE, i.e. chi <= 27
 * for qutrits and chi <= 40 for qubits; a larger shape returns GCAMPS_ESIZE and launches nothing.
 *
 * Every pointer is device memory of the current device, owned by the caller.  theta_dev: chi_l x d
 * x d x chi_r complex entries (interleaved re, im; row-major over (a, s, t, b)).  s2_dev, vn_dev:
 * K = gcamps_num_candidates(d) doubles each, the Renyi-2 and von Neumann entropies of every class
 * as in gcamps_score_theta.  choice_dev: 3 int32, the class the von Neumann disentangler (score_kind 0,
 * rank threshold of cutoff 0) would apply (0 = none; a class is applied only if it lowers the entropy by
 * more than tie_tol, ties to the lowest index; handles made with score_kind 1 or 2 can choose otherwise),
 * the number of exact entropies its Renyi-2 pruning evaluated, and the device status of the call
 * (0 or a GCAMPS_E* code; the eigenvalue search runs a fixed number of steps, so 0 in practice).  cuda_stream: the cudaStream_t
 * to run on, NULL for the default stream.  Asynchronous: the outputs are valid once the stream has
 * passed this call.
 *
 * The first call on a device, with that device current, does a one-time set-up: it looks up the
 * device address of the static array and copies the class tables into static device memory
 * (synchronous copies).  Make that first call before any stream capture.  All calls on a device
 * share the one array and it keeps the last call's contents; each call clears the words that must
 * start at zero itself.  Calls whose kernels overlap on the GPU (several streams, or several host
 * threads at once) race on the array and give wrong results: serialise them.
 * Returns GCAMPS_OK; GCAMPS_EINVAL (d not 2 or 3, a null pointer, chi < 1, tie_tol < 0 or NaN);
 * GCAMPS_ESIZE; GCAMPS_ECUDA (set-up or launch failed). */
#define GCAMPS_NOALLOC_MAX_SIDE 81
int gcamps_score_theta_noalloc(int d, int chi_l, int chi_r, const double* theta_dev, double* s2_dev,
                               double* vn_dev, int32_t* choice_dev, double tie_tol, void* cuda_stream);

/* Measured arithmetic peaks of the current GPU, the denominators of the engine's roofline (no counterpart in
 * the paper): tflops[0] FP64 fused multiply-add, tflops[1] FP32 fused multiply-add, tflops[2] FP64
 * tensor-core MMA (m8n8k4), in TFLOP/s counting 2 flops per multiply-add, from CUDA-event timings of grids
 * of independent chains (under about a second each; one small allocation).  count: entries of tflops
 * (>= 3).  Synchronising. */
int gcamps_measure_peaks(double* tflops, int count);

/* Wait for all enqueued work; returns the sticky device status of circuit 0..batch-1 folded.  No
 * counterpart in the paper. */
int gcamps_sync(gcamps_t* h);
/* Back to |0...0>, C = I (the initial state of Sec. 2.2), counters and decisions cleared, for every
 * circuit (enqueued on the handle's stream; asynchronous). */
int gcamps_reset(gcamps_t* h);
/* Message of the handle's most recent failed call ("" if none has failed, "null handle" for NULL);
 * owned by the handle, valid until its next failing call or gcamps_destroy.  No counterpart in the
 * paper. */
const char* gcamps_last_error(gcamps_t* h);

#ifdef __cplusplus
}
#endif
#endif /* GCAMPS_H_INCLUDED */
