/*
 * qcd_gb300.h -- C ABI of the Clover-Wilson SAP-BiCGStab quark solver for
 * NVIDIA GB300 (sm_103a).
 *
 * The library implements the quark solver of arXiv:2109.10687:
 *   D = 1 + C - kappa H                          (App. A)
 *   A = C_inv D = I - kappa C_inv H              (Sec. 3, Eq. hoppingmat)
 * preconditioned by the red/black Schwarz alternating procedure with Jacobi
 * domain inverses (Sec. 3, Eq. Msap, Algorithms 1-3), solved by BiCGStab
 * (Algorithm 5) inside a float64 defect-correction loop (Algorithm 4).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every function returns an int status (QCD_OK = 0 on success).  No C++
 *   exception crosses this boundary.  qcd_last_error() gives a message for
 *   the last failing call on a context.
 * - dims[4] = {Lx, Ly, Lz, Lt}; domain[4] = {dx, dy, dz, dt}.  Every d_mu is a
 *   power of two, dx*dy*dz*dt <= 256, and every L_mu is a multiple of 2*d_mu
 *   (an even number of domains per direction keeps the red/black colouring
 *   of Sec. 3 consistent across the periodic boundary).  Default domain 4^4.
 *   The domains are the blocks the fields are stored in and, by default, the
 *   SAP domains; qcd_set_sap_domain gives the SAP domains of any extents.
 * - Boundary conditions: periodic in x, y, z; bc_t = +1 (periodic) or -1
 *   (antiperiodic) in t, applied as a sign on every hop across t = Lt-1 <-> 0.
 * - CANONICAL layout (host or device, float64, little endian, x fastest):
 *     quark field : [t][z][y][x][colour 3][spin 4][re, im]        (Sec. 4, "K")
 *     gauge field : [t][z][y][x][mu 4 = x,y,z,t][row 3][col 3][re, im]
 *   With nrhs > 1 right-hand sides the quark fields are stacked: [rhs][...].
 * - Gamma basis of canonical quark fields: QCD_BASIS_CHIRAL (default;
 *   gamma_5 = diag(1,1,-1,-1)) or QCD_BASIS_PAPER (the matrices printed in
 *   App. A).  Kernels always work in the chiral basis; paper-basis fields are
 *   rotated on import and export.
 * - INTERNAL layout: the device-resident, domain-blocked structure of arrays
 *   used by the kernels.  Its size comes from qcd_field_bytes(); the caller
 *   allocates such buffers (cudaMalloc, torch, ...) and owns them; the
 *   library only reads and writes them on the given stream.  Fields move
 *   between the two layouts with qcd_import_spinor / qcd_export_spinor.
 * - Precision codes: QCD_PREC_DOUBLE (float64 storage and arithmetic),
 *   QCD_PREC_SINGLE (float32), QCD_PREC_HALF (float16 storage with a float32
 *   norm per site; float32 arithmetic).
 * - stream: a cudaStream_t passed as void*; NULL is the legacy default stream.
 *   Calls that return host-visible results (qcd_solve, qcd_norm2, ...)
 *   synchronise that stream before returning.
 * - The library owns its copies of U, the clover term and its workspaces
 *   (device memory it allocates on first use and frees in qcd_destroy).
 * - A context is not thread safe; use one context per host thread.
 */
#ifndef QCD_GB300_H
#define QCD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum qcd_status {
  QCD_OK = 0,
  QCD_ERR_ARG = 1,            /* invalid argument or unsupported size       */
  QCD_ERR_CUDA = 2,           /* a CUDA runtime call failed                 */
  QCD_ERR_OOM = 3,            /* device allocation failed                   */
  QCD_ERR_NOT_CONVERGED = 4,  /* iteration limit reached before tolerance   */
  QCD_ERR_BREAKDOWN = 5,      /* BiCGStab breakdown (rho, <r~|q> or |t|^2=0) */
  QCD_ERR_NONFINITE = 6,      /* NaN or Inf met in a residual              */
  QCD_ERR_TIMEOUT = 7,        /* a bounded device-side wait gave up         */
  QCD_ERR_STATE = 8           /* call out of order (no gauge field, ...)    */
};

enum qcd_precision {
  QCD_PREC_DOUBLE = 0,
  QCD_PREC_SINGLE = 1,
  QCD_PREC_HALF = 2,
  QCD_PREC_HALF_GAUGE = 3  /* SAP only: float16 links and C_inv, float32 vectors */
};
enum qcd_basis { QCD_BASIS_CHIRAL = 0, QCD_BASIS_PAPER = 1 };

typedef struct qcd_ctx qcd_ctx;

/* Parameters of qcd_solve (Algorithms 4 and 5). */
typedef struct qcd_solve_params {
  double tol;          /* outer stop: |b - D x| / |b| < tol, float64 (Alg. 4)  */
  double inner_tol;    /* inner stop of Algorithm 5 on the preconditioned
                          system, relative to its right-hand side            */
  int max_outer;       /* defect-correction steps (Alg. 4), e.g. 20          */
  int max_inner;       /* BiCGStab iterations per inner solve (Alg. 5)      */
  int n_sap;           /* loop count of Algorithm 1 (K applied n_sap+1 times) */
  int n_jac;           /* A_EE applications in Algorithm 2 (>= 1)            */
  int sap_prec;        /* SAP storage: QCD_PREC_SINGLE, QCD_PREC_HALF (links,
                          C_inv and vectors) or QCD_PREC_HALF_GAUGE (links
                          and C_inv only)                                    */
  int use_graph;       /* 0: kernels launched one by one; 1: each half of a
                          BiCGStab iteration replayed as a CUDA graph; 2: the
                          whole inner loop as one graph with a conditional
                          while node (no host round trip per iteration)      */
  int x_is_guess;      /* 1: x holds an initial guess on entry (resume)      */
  int residual_prec;   /* precision of x, r = b - D x and D in Algorithm 4:
                          0 double-float (default: two float32, ~48 bits,
                          on the float32 pipes, which on this GPU are far
                          wider than the float64 ones; the residual it
                          stops on is within 2^-48 (1 + 300 |x| / |b|) of
                          the float64 residual of the same x), 1 native
                          float64; other values QCD_ERR_ARG.  The flexible
                          GMRES outer iteration computes in native float64
                          either way; the shared-launch batch solve keeps x,
                          r and b in float64 and computes D x as selected.  */
  int outer_restart;   /* outer iteration: 0 (default) the defect correction
                          of Algorithm 4; m >= 1 flexible GMRES with restart
                          length m, in float64, each inner SAP-BiCGStab
                          solve acting as a preconditioner that may change
                          from step to step (the flexible outer solver Sec. 3
                          names as an alternative to Algorithm 4; max_outer
                          then counts its steps).  Requires nrhs = 1, else
                          QCD_ERR_ARG.                                       */
} qcd_solve_params;

/* Results of qcd_solve, one entry per right-hand side where indicated. */
typedef struct qcd_solve_info {
  int outer_iters;         /* outer steps taken (defect-correction or
                              flexible GMRES steps)                        */
  int inner_iters;         /* BiCGStab iterations summed over outer steps  */
  int status;              /* qcd_status of the solve                      */
  double true_resid;       /* largest final |b - D x| / |b| over the rhs   */
  double seconds;          /* wall time inside qcd_solve                   */
} qcd_solve_info;

/* ---- context ---------------------------------------------------------- */

/* Create a context for one lattice on the current CUDA device.
 * dims, domain: see above (domain may be NULL for 4^4).  bc_t: +1 or -1.
 * basis: QCD_BASIS_CHIRAL or QCD_BASIS_PAPER for canonical quark fields.
 * Errors: QCD_ERR_ARG (bad sizes), QCD_ERR_CUDA, QCD_ERR_OOM. */
int qcd_create(const int dims[4], const int domain[4], int bc_t, int basis, qcd_ctx** out);

/* Free every device buffer the context owns, then the context. */
int qcd_destroy(qcd_ctx* ctx);

/* Message of the last failing call on ctx (or, when ctx is NULL, of the
 * calling thread's last failing qcd_create).  The string is owned by the
 * library and stays valid until the next failing call on ctx (or the
 * thread's next failing qcd_create). */
const char* qcd_last_error(const qcd_ctx* ctx);

/* Library version string, e.g. "qcd_gb300 1.0". */
const char* qcd_version(void);

/* ---- gauge field and clover term -------------------------------------- */

/* Copy the gauge field U (canonical layout, float64, 4 V 9 complex) into the
 * context in float64, float32 and float16 internal layouts.  U_mu(n) is the
 * SU(3) link from n to n + mu (App. A; U_{-mu}(n) = U_mu(n - mu)^dag).
 * on_device: 1 if U is a device pointer, 0 for host memory.
 * check_tol > 0: reject links with |U^dag U - 1| or |det U - 1| above it
 * (QCD_ERR_ARG).  Invalidates a previously built clover term. */
int qcd_set_gauge(qcd_ctx* ctx, const double* U, int on_device, double check_tol, void* stream);

/* Set the hopping parameter kappa and the clover coefficient c_SW (App. A).
 * Invalidates a previously built clover term. */
int qcd_set_params(qcd_ctx* ctx, double kappa, double csw);

/* Build the clover term of App. A from the four-leaf field strength
 *   F_mu,nu = (Q_mu,nu - Q_mu,nu^dag) / 8,
 *   C = i kappa c_SW sum_{mu<nu} sigma_mu,nu F_mu,nu,
 * as two 6x6 Hermitian chiral blocks per site, and C_inv = (1 + C)^-1
 * (float64 arithmetic; float64, float32 and float16 copies are kept).
 * Errors: QCD_ERR_STATE without a gauge field; QCD_ERR_NONFINITE if a block
 * is singular. */
int qcd_build_clover(qcd_ctx* ctx, void* stream);

/* ---- fields ----------------------------------------------------------- */

/* Bytes of one internal quark field of the given precision times nrhs. */
int qcd_field_bytes(const qcd_ctx* ctx, int prec, int nrhs, size_t* bytes);

/* Canonical float64 (host or device) -> internal layout of precision prec.
 * A host buffer (src_on_device = 0 / dst_on_device = 0) in page-locked
 * memory is read or written by the conversion kernel itself through its
 * mapped device address; pageable memory goes through a temporary device
 * copy.  With a host buffer both calls return after the transfer is
 * complete, so the buffer may be reused at once. */
int qcd_import_spinor(qcd_ctx* ctx, void* dst, const double* src, int prec, int nrhs,
                      int src_on_device, void* stream);

/* Internal layout of precision prec -> canonical float64 (host or device). */
int qcd_export_spinor(qcd_ctx* ctx, double* dst, const void* src, int prec, int nrhs,
                      int dst_on_device, void* stream);

/* ---- operators (all on internal-layout device buffers) ---------------- */

/* out = D in (dagger = 0) or D^dag in = gamma_5 D gamma_5 in (dagger = 1),
 * D x = (1 + C) x - kappa sum_mu [(1 - g_mu) U_mu(n) x(n+mu)
 *                                + (1 + g_mu) U_mu(n-mu)^dag x(n-mu)]   (App. A).
 * prec: QCD_PREC_DOUBLE or QCD_PREC_SINGLE.  out and in must not alias.
 * The operator kernel is launched with programmatic stream serialization:
 * it may start while the previous kernel on the stream drains and waits for
 * that kernel's completion before it reads anything (back-to-back calls
 * overlap their tails).  The first call for a given nrhs and precision
 * times the compiled launch shapes (see qcd_set_tuning). */
int qcd_apply_D(qcd_ctx* ctx, void* out, const void* in, int prec, int dagger, int nrhs,
                void* stream);

/* out = A in = in - kappa C_inv H in (Sec. 3, Eq. hoppingmat); float32. */
int qcd_apply_A(qcd_ctx* ctx, void* out, const void* in, int nrhs, void* stream);

/* out = (1 + C) in (inverse = 0) or C_inv in (inverse = 1); prec DOUBLE or
 * SINGLE.  out may alias in. */
int qcd_apply_clover(qcd_ctx* ctx, void* out, const void* in, int prec, int inverse, int nrhs,
                     void* stream);

/* One block of A restricted to a domain colour (Sec. 3): row, col in {0 = E,
 * 1 = O}.  out (all sites) = A_rc in: sites of colour row receive the
 * result, the others are set to zero.  float32; test and diagnostic use. */
int qcd_apply_A_block(qcd_ctx* ctx, void* out, const void* in, int row, int col, void* stream);

/* x = M_SAP b (with_A = 0, Algorithm 1) or x = A M_SAP b (with_A = 1,
 * Algorithm 3) on float32 internal fields; sap_prec = QCD_PREC_SINGLE keeps
 * everything in float32, QCD_PREC_HALF stores links, C_inv and the sweep
 * vectors in float16, QCD_PREC_HALF_GAUGE only links and C_inv.
 * n_sap >= 0 is the loop count of Algorithm 1; n_jac >= 1 the number of
 * A_EE applications of Algorithm 2.  out and in must not alias. */
int qcd_sap_apply(qcd_ctx* ctx, void* out, const void* in, int n_sap, int n_jac, int sap_prec,
                  int with_A, void* stream);

/* SAP domains independent of the context's storage blocking (Sec. 3; the
 * paper's runs use 16x6x4x3 to 16x12x8x12 domains, Tables 2-3).  sdom[4]:
 * extents of any size (not only powers of two) with every L_mu a multiple
 * of 2 sdom_mu, and at most 1152 sites per domain or at most 8 time slices
 * (sdom_t <= 8) of at most 448 sites (sdom_x sdom_y sdom_z <= 448); NULL
 * returns to the storage domains (the default).  With such domains every
 * SAP application (qcd_sap_apply, qcd_sap_apply_nrhs, qcd_solve) runs
 * Algorithms 1-2 on them with a kernel that holds one domain per CTA in
 * shared memory (x and s in float32, links and C_inv read from the internal
 * layouts; domains up to 1152 sites) or, with float16 links and C_inv, one
 * thread-block cluster per domain (see qcd_set_sap_shape); sap_prec must be
 * QCD_PREC_SINGLE or QCD_PREC_HALF_GAUGE, and QCD_PREC_HALF_GAUGE with the
 * cluster shape for domains above 1152 sites (QCD_ERR_ARG otherwise, at the
 * SAP call).  Errors: QCD_ERR_ARG for a domain that fits neither kernel. */
int qcd_set_sap_domain(qcd_ctx* ctx, const int sdom[4]);

/* qcd_sap_apply for nrhs stacked fields (in and out hold nrhs internal
 * float32 fields one after the other).  With 4^4 domains every right-hand
 * side goes through each block-kernel launch and shares its staged links and
 * C_inv, as in the batched qcd_solve; each right-hand side's result is the
 * one qcd_sap_apply gives for it alone.  1 <= nrhs <= 65535, else
 * QCD_ERR_ARG. */
int qcd_sap_apply_nrhs(qcd_ctx* ctx, void* out, const void* in, int nrhs, int n_sap, int n_jac, int sap_prec,
                       int with_A, void* stream);

/* ---- BLAS-1 (float32 internal fields, float64 results) --------------- */

/* *result = |a|^2 (host pointer), accumulated per block in float32 and
 * across blocks in float64, in a fixed order (deterministic). */
int qcd_norm2(qcd_ctx* ctx, double* result, const void* a, int prec, int nrhs, void* stream);

/* |a|^2 like qcd_norm2, for callers that must not allocate device memory
 * during the call -- for example code running under a caching allocator or
 * memory pool that owns all free device memory, or code that must not
 * trigger the implicit device synchronisation a cudaMalloc can cause.  The
 * paper has no counterpart; this is an interface convenience.
 * The call allocates nothing: no cudaMalloc, cudaFree or allocating library
 * routine.  Its scratch (per-block partial sums, completion counters and
 * results) is a static device array of about 514 KB inside the library,
 * held by every GPU that loads the library until the process exits.  Limits:
 * 1 <= nrhs <= 16 (QCD_ERR_ARG otherwise).  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress) with that
 * device current.  Every
 * call shares the one array: calls whose work overlaps on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * result: host pointer, nrhs doubles; a: internal-layout field of precision
 * SINGLE or DOUBLE.  Synchronises the stream. */
int qcd_norm2_noalloc(qcd_ctx* ctx, double* result, const void* a, int prec, int nrhs, void* stream);

/* result[0] + i result[1] = <a|b> = a^dag b (host pointer). */
int qcd_cdot(qcd_ctx* ctx, double result[2], const void* a, const void* b, int prec, int nrhs,
             void* stream);

/* ---- solver ----------------------------------------------------------- */

/* Solve D x = b for nrhs right-hand sides (canonical float64 fields, host
 * memory when on_device = 0, device memory when 1).  Algorithm 4 in float64
 * (or flexible GMRES, see outer_restart) around Algorithm 5 in float32 on
 * (A M_SAP) y = C_inv r / |r|, the SAP preconditioner in float32 or float16
 * storage.  With nrhs > 1 all right-hand
 * sides advance together and share every gauge-field and clover load.
 * Returns QCD_OK when every rhs reached tol, QCD_ERR_NOT_CONVERGED,
 * QCD_ERR_BREAKDOWN or QCD_ERR_NONFINITE otherwise (x then holds the last
 * iterate).  info may be NULL. */
int qcd_solve(qcd_ctx* ctx, double* x, const double* b, int nrhs, int on_device,
              const qcd_solve_params* params, qcd_solve_info* info, void* stream);

/* Fill params with defaults: tol 1e-10, inner_tol 1e-6, max_outer 20,
 * max_inner 500, n_sap 4, n_jac 4, sap_prec SINGLE, use_graph 0,
 * x_is_guess 0, residual_prec 0 (double-float), outer_restart 0 (Algorithm 4). */
int qcd_solve_params_default(qcd_solve_params* params);

/* ---- ragged batches of lattices --------------------------------------- */

typedef struct qcd_batch qcd_batch;

/* Group n contexts (lattices that may differ in size, gauge field, kappa and
 * c_SW; all on one device) for batched calls.  The batch does not own the
 * contexts; destroy it before them. */
int qcd_batch_create(int n, qcd_ctx* const* ctxs, qcd_batch** out);
int qcd_batch_destroy(qcd_batch* batch);
const char* qcd_batch_last_error(const qcd_batch* batch);

/* out[i] = D_i in[i] (dagger = 0) or D_i^dag in[i] for every lattice of the
 * batch in ONE kernel launch (float32 internal-layout fields of each
 * context; App. A).  A work list gives each lattice a contiguous range of
 * blocks. */
int qcd_batch_apply_D(qcd_batch* batch, void* const* out, const void* const* in, int dagger, void* stream);

/* Solve D_i x_i = b_i for every lattice (one right-hand side each, canonical
 * float64 fields as in qcd_solve; Algorithm 4 around Algorithm 5 on
 * A M_SAP, Sec. 3).  When every lattice has 4^4 domains (and no SAP domains
 * of its own, see qcd_set_sap_domain) and outer_restart = 0, the lattices
 * are solved in SHARED LAUNCHES (x, r and b in float64; D x of the
 * residual in double-float for residual_prec 0, in float64 for 1): each
 * SAP half-sweep (Algorithm 1), each application of A and of the float64 D,
 * and each fused BLAS-1 step of Algorithm 5 is one kernel launch over every
 * lattice, through work lists built on the first call; the inner loop is one
 * CUDA graph with a conditional while node (use_graph = 2; otherwise the
 * kernels are launched one by one), run while any lattice iterates.  A
 * lattice that has converged stops there while the others continue; per
 * lattice the iterations and the float64 true residual are those of its own
 * Algorithm 4/5.  The batch allocates its buffers on the first call (about
 * 1.5 KB per site over all lattices) and keeps them.  Other batches (or
 * after qcd_batch_set_shared(batch, 0)) run the lattices' solves at the same
 * time on one stream each, so that their kernels interleave.  Both forms
 * are ordered after `stream`.  infos (may be NULL) receives one record per
 * lattice (seconds: the whole batch); returns the first failing lattice's
 * status, QCD_OK if all met params->tol. */
int qcd_batch_solve(qcd_batch* batch, double* const* x, const double* const* b, int on_device,
                    const qcd_solve_params* params, qcd_solve_info* infos, void* stream);

/* 1 (default): qcd_batch_solve uses shared launches where it can; 0: always
 * the concurrent per-lattice solves. */
int qcd_batch_set_shared(qcd_batch* batch, int enable);

/* ---- gradients -------------------------------------------------------- */

/* Gradient of L = Re(eta^dag D^-1 b) (canonical float64 fields on the
 * device):
 *   grad_b = D^-dag eta = gamma_5 D^-1 gamma_5 eta            (solve),
 *   grad_U[n][mu] = G_mu(n), with dL = sum Re tr(G^dag dU), from the
 *   hopping term (outer products of x = D^-1 b and lambda = grad_b) and the
 *   clover leaves; with project = 1 grad_U holds TA(G U^dag) instead, the
 *   su(3) projection (traceless anti-Hermitian part).
 * x and lam may be supplied (non-NULL, canonical float64 device fields) to
 * skip the two solves; otherwise they are solved with params (when both are
 * needed and params->outer_restart = 0, as the two right-hand sides b and
 * gamma_5 eta of one batched solve).
 * grad_U layout: canonical gauge layout. */
int qcd_grad(qcd_ctx* ctx, const double* eta, const double* b, const double* x,
             const double* lam, double* grad_b, double* grad_U, int project,
             const qcd_solve_params* params, void* stream);

/* ---- instrumentation -------------------------------------------------- */

enum qcd_kernel_class {
  QCD_KC_DSLASH = 0,     /* D / D^dag / A applies                      */
  QCD_KC_SAP_BLOCK = 1,  /* SAP domain kernels (Algorithms 1-3)        */
  QCD_KC_BLAS = 2,       /* fused BLAS-1 and reductions                */
  QCD_KC_DOUBLE = 3,     /* float64 operator and defect correction    */
  QCD_KC_OTHER = 4,
  QCD_KC_COUNT = 5
};

/* enable = 1: bracket every kernel launch with CUDA events on its stream
 * and accumulate per-class device time; 0: stop (the default). */
int qcd_profile_enable(qcd_ctx* ctx, int enable);

/* Per class: launches and summed device milliseconds since the last reset
 * (synchronises the events).  reset = 1 clears the counters afterwards. */
int qcd_profile_read(qcd_ctx* ctx, int kernel_class, long long* launches, double* ms, int reset);

/* Launch-shape autotuning (on by default).  With tuning on, the first call of
 * a tunable kernel for a given key times each compiled shape on the real
 * arguments and keeps the fastest; the shapes change scheduling only, not
 * the arithmetic.  Tunable: the float32 D / D^dag / A operator (threads per
 * block, blocks per SM; key: right-hand sides) and the SAP block kernel of
 * 4^4 domains (sites per thread; key: SAP storage, lattice, right-hand
 * sides, n_sap, n_jac -- the whole M_SAP of Algorithm 1 is timed in each
 * shape).  A solve tunes before it captures its inner loop in a graph.
 * enable = 0 turns tuning off and forgets the choices (the default shape is
 * then used). */
int qcd_set_tuning(qcd_ctx* ctx, int enable);

/* Links of the float32 D, D^dag and A (App. A) as 12 reals: an SU(3)
 * matrix is fixed by its first two rows (the third is the complex conjugate
 * of their cross product), so the HBM-bound operator can read 48 instead of
 * 72 bytes per link and rebuild the third row.  mode -1 (default): 12
 * reals whenever the links given to qcd_set_gauge are SU(3) to 1e-9; 0:
 * never; 1: always (an operator call then returns QCD_ERR_STATE if the
 * links are not SU(3) to 1e-9).  The format is fixed by this setting and
 * the links, not by the autotuner, whose launch shapes stay bit-identical;
 * the rebuilt row differs from the stored float32 one by float32 rounding.
 * QCD_ERR_ARG for other values. */
int qcd_set_link_compression(qcd_ctx* ctx, int mode);

/* *reals = 12 or 18: the link format the float32 operators (single and
 * batched) use now, as qcd_set_link_compression and the links decide.
 * QCD_ERR_ARG for null arguments. */
int qcd_link_format(const qcd_ctx* ctx, int* reals);

/* Fix the SAP kernel's shape: -1 autotuned (default).  For 4^4 domains:
 * 0 one site per thread (256 threads per domain), 1 two sites per thread
 * (128 threads per domain, each thread two independent site streams), 2 one
 * site per thread and one CTA per domain and right-hand side (with nrhs > 1;
 * each CTA stages the domain's links and C_inv itself, instead of running
 * every right-hand side through one staged copy), 3 the whole M_SAP
 * (Algorithm 1, all 2 (n_sap + 1) half-sweeps) in one launch of resident
 * CTAs that take (half-sweep, domain) items in order and wait, bounded, for
 * the eight neighbouring domains of the previous half-sweep through
 * per-domain flags instead of for a whole grid, 4 as 3 with half of the
 * CTAs starting 10 us later; every shape computes the same M_SAP bit for
 * bit.  For domains set with qcd_set_sap_domain and float16 links and C_inv
 * (QCD_PREC_HALF_GAUGE): 0 one thread-block cluster per domain, one CTA per
 * time slice (at most 8 slices of at most 448 sites), links and C_inv staged
 * in shared memory and the time hops between slices through distributed
 * shared memory; 1 to 4 one CTA per domain reading links and C_inv through
 * L1.  QCD_ERR_ARG for other values. */
int qcd_set_sap_shape(qcd_ctx* ctx, int shape);

/* Autotuner over SAP domain shapes, by time to solution.  The domain shape
 * fixes a context's field layout, so for each candidate this creates a
 * temporary context (dims, domain = candidate, bc_t, basis as qcd_create),
 * sets U, kappa, c_SW, builds the clover term, solves D x = b once to warm
 * it and once more timed (params as qcd_solve; NULL: defaults), and
 * destroys it.  U and b are canonical float64 fields, both on the device
 * (on_device = 1) or both in host memory.  candidates: n shapes of 4 ints;
 * n = 0 (candidates may be NULL) takes the built-in list (4^4, 8x4x4x2,
 * 2x4x4x8, 4x4x2x4, 8x8x2x2, 4x4x4x2, 2^4; qcd_tune_domain_default_count()
 * of them).  A candidate that does not fit the lattice (see qcd_create) or
 * whose solve does not reach params->tol is skipped.  best_domain receives
 * the fastest shape; seconds (NULL, or one double per candidate) the timed
 * solve of each, -1 for a skipped one.  Returns QCD_ERR_ARG if no candidate
 * solved.  Allocates a temporary x (one field) and each candidate's context;
 * synchronises the device's default stream. */
int qcd_tune_domain(const int dims[4], int bc_t, int basis, const double* U, const double* b, int on_device,
                    double kappa, double csw, const qcd_solve_params* params, const int* candidates, int n,
                    int best_domain[4], double* seconds);
int qcd_tune_domain_default_count(void);

/* Text report of the tuned choices, one line per key:
 * "<key> <shape> <ms>", followed by the time of every shape tried. */
int qcd_tuning_report(qcd_ctx* ctx, char* buf, size_t len);

/* Number of kernels the library has launched on this context so far. */
int qcd_launch_count(const qcd_ctx* ctx, long long* count);

/* ---- failure detection ------------------------------------------------- */

/* Device status word: kernels record device-side failures here, e.g.
 * QCD_ERR_TIMEOUT when the SAP block kernel's bounded wait for its staging
 * copies gives up (the kernel then waits once more, also bounded, and
 * returns; the context stays usable).  qcd_solve checks the word after every
 * inner solve and returns its code.  *status = the word (QCD_OK if no failure);
 * reset = 1 clears it.  Synchronises the stream. */
int qcd_device_status(qcd_ctx* ctx, int* status, int reset, void* stream);

/* Test hooks for the failure paths (the paper has no counterpart).  what:
 * QCD_INJECT_NONE clears; QCD_INJECT_STAGING_WAIT makes the SAP block
 * kernel's staging wait expect 16 bytes more than its copies bring, so the
 * bounded wait runs out (about a second) and the kernel records
 * QCD_ERR_TIMEOUT; QCD_INJECT_HALO_WAIT does the same to its wait for the
 * face-halo copy (launches with a surface term).  No GPU fault is
 * involved. */
enum { QCD_INJECT_NONE = 0, QCD_INJECT_STAGING_WAIT = 1, QCD_INJECT_HALO_WAIT = 2 };
int qcd_test_inject(qcd_ctx* ctx, int what);

/* Measurement utility (no counterpart in the paper): the device's float32
 * FMA throughput in TFLOP/s (2 flop per FMA), from a kernel of independent
 * fused multiply-add chains over every SM, timed with CUDA events on
 * `stream` (the best of three launches after a warm-up).  It is the
 * denominator of the ALU roofline of the SAP block kernel.  Synchronises the
 * stream; writes *tflops.  QCD_ERR_ARG for null pointers, QCD_ERR_CUDA on a
 * CUDA error. */
int qcd_measure_fp32_peak(qcd_ctx* ctx, double* tflops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* QCD_GB300_H */
