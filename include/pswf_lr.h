/*
 * pswf_lr.h -- C-ABI of the PSWF-LR reciprocal-space evaluation on B300.
 *
 * What is computed (paper: "Prolate spheroidal wave functions enable fast
 * and exponent-aware long-range machine learning interatomic potentials"):
 * for a periodic orthorhombic box of volume V, N atoms at r_i and K latent
 * charge channels q_i^(c), each with its own exponent p_c in 1..6,
 *
 *   E_c = 1/(2V) sum_{k != 0} Phi-hat_{p_c}(k) |rho^(c)(k)|^2 + E^{0,(p_c)}
 *                                                   (Eq. Fourier)
 * evaluated by PSWF spreading on a uniform grid, a batched 3-D FFT, the
 * mollified multiplier W-hat(k)^-2 Phi-hat_p(k) and the inverse FFT
 * (Methods, "Accelerating atom-grid spreading with PSWFs", Eq. EthetaLR,
 * steps (i)-(iv)), then the gather of per-atom potentials
 * phi_i^(c) = dE/dq_i^(c) and forces F_i = -dE/dr_i.
 * Phi-hat_p is Eq. (PhiH); E^{0,(p)} is the zero-frequency correction of
 * "Implementation details" (Eq. Correction and the p > 3 formula); the
 * self-energy E_self^(p) of the same section is returned separately.
 * Hyperparameters follow "Parameter selection".
 *
 * Conventions for every entry point:
 *  - Return 0 (PSWF_OK) or a negative PSWF_E* status; nothing throws and no
 *    entry point aborts the process.  pswf_strerror() names a status and
 *    pswf_plan_last_error() gives the plan's last message.
 *  - "device" pointers are CUDA global memory on the plan's device, owned by
 *    the caller; "host" pointers are ordinary CPU memory owned by the caller.
 *  - Work is enqueued on the plan's CUDA stream; only calls documented as
 *    synchronising wait for it.
 *  - Lengths are Angstrom; energies are in q^2 / Angstrom^p (Coulomb
 *    constant 1).
 *  - Real arrays on the device are float (precision 0, FP32 path) or double
 *    (precision 1, FP64 path) as chosen at plan creation ("real" below).
 */
#ifndef PSWF_LR_H
#define PSWF_LR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define PSWF_OK 0
#define PSWF_EINVAL (-1)           /* bad argument (p outside 1..6, box <= 0, n > n_max, ...) */
#define PSWF_ENOMEM (-2)           /* device allocation failed or workspace too small */
#define PSWF_ECUFFT (-3)           /* a cuFFT call failed */
#define PSWF_ECUDA (-4)            /* a CUDA runtime call or kernel launch failed */
#define PSWF_ETIMEOUT (-5)         /* a bounded wait ran out (pswf_sync_for, pswf_server_wait_for) */
#define PSWF_ENONFINITE (-6)       /* NaN or Inf in the positions */
#define PSWF_ETOLUNREACHABLE (-7)  /* grid too coarse for the mollifier band (h k_c >= pi) */
#define PSWF_ESTATE (-8)           /* call out of order (e.g. execute before set_points) */
#define PSWF_ECELL (-9)            /* real space: a cell of the cell list holds more than 2048 atoms */
#define PSWF_EBOUNDS (-10)         /* bounds-checked build only: a kernel index left its buffer (access skipped) */

/* ---- options ----------------------------------------------------------- */
#define PSWF_FLAG_BACKWARD 1       /* reserve a second grid so pswf_backward can run */
#define PSWF_FLAG_VIRIAL 2         /* pswf_execute also reduces the virial tensor (pswf_virial, pswf_stress) */
#define PSWF_FLAG_REAL_SPACE 4     /* reserve the real-space complement's cell list (pswf_real_space) */

typedef struct {
  double tol;      /* target LR tolerance eps_tot (default 1e-5) */
  double r_c;      /* mollifier cutoff r_c in Angstrom (required, > 0) */
  double c;        /* mollifier bandwidth; 0 -> log(3 / tol) ("Parameter selection") */
  double c_w;      /* window bandwidth; 0 -> P pi (1 - eta / 2) */
  double eta;      /* Nyquist factor of h <= eta pi / k_c; 0 -> 0.5 */
  int P;           /* stencil width per dimension; 0 -> smallest meeting tol / 3 */
  int grid[3];     /* grid points per dimension; 0 -> ceil(L / h) rounded to 2^a 3^b 5^c 7^d */
  int precision;   /* 0: FP32 spread/FFT/interp (FP64 tables and reductions); 1: all FP64 */
  int flags;       /* PSWF_FLAG_* */
} pswf_opts;

typedef struct {
  double c, c_w, r_c, k_c, eta, tol;
  double est_err_spread;   /* planner's estimate of the spreading error */
  double est_err_band;     /* psi_0^c(1), size of the band truncation */
  double lambda0, C0;      /* eigenvalue lambda_0 of psi_0^c and C_0 = int_0^1 psi_0^c */
  double box[3], h[3];
  int grid[3];
  int P, K, precision, deg_window, deg_mult, flags;
  int64_t n_max;
  int64_t workspace_bytes; /* device bytes pswf_plan_set_workspace wants */
  int B;                   /* structures per call (1 for single-structure plans) */
  int batch;               /* 1 for plans made by pswf_batch_plan_create */
  int transform;           /* pswf_plan_info: PSWF_TRANSFORM_* of the plan (0 from pswf_plan_params) */
  int nkx;                 /* pruned transforms: x frequencies 0..nkx-1 kept (others are out of band) */
  double cell[9];          /* pswf_plan_info: lattice vectors as rows (diag(box) for a box; box_max for
                              batch plans); box[] then holds the edge lengths |a_d| */
  int deg_real;            /* degree of the real-space mollifier pieces G_p (pswf_real_space) */
} pswf_info;

/* Transform of a plan.  FULL: cuFFT 3-D real transforms of every structure
 * slot.  PRUNED: single-structure plans whose band |k| < k_c reaches only
 * kx < nkx <= 3/4 (Mx/2 + 1): 1-D transforms along x, then 2-D (z, y)
 * transforms of the nkx planes only (cuFFT).  PRUNED_X: the same with the
 * x passes done by this library's kernels (FP32, Mx = 32 N1 with
 * 2 <= N1 <= 16), which write and read only the nkx planes.  OWN: when My
 * and Mz are of that form too, every pass is this library's: x, z, then the
 * multiplier fused with the y transforms, z and x back. */
#define PSWF_TRANSFORM_FULL 0
#define PSWF_TRANSFORM_PRUNED 1
#define PSWF_TRANSFORM_PRUNED_X 2
#define PSWF_TRANSFORM_OWN 3

typedef struct pswf_plan_s* pswf_plan;

/* Fills *o with the defaults above (r_c left at 0: the caller must set it). */
void pswf_opts_default(pswf_opts* o);

/* Host-only parameter selection ("Parameter selection"): runs the planner
 * without touching a GPU and fills *out (n_max and workspace_bytes are 0).
 * box: host [3] edge lengths; p: host [K] exponents in 1..6; opts: host,
 * required (r_c has no default).  Returns PSWF_EINVAL or
 * PSWF_ETOLUNREACHABLE on bad input. */
int pswf_plan_params(const double box[3], int K, const int* p, const pswf_opts* opts, pswf_info* out);

/* Creates a plan for up to n_max atoms on the current CUDA device: runs the
 * planner (the hyperparameters of "Parameter selection": c from the
 * tolerance, grid spacing h <= eta pi / k_c with k_c = c / r_c, the stencil
 * width P and window bandwidth c_w of "Accelerating atom-grid spreading with
 * PSWFs"), builds the batched cuFFT plans (no cuFFT allocation) and records
 * the stream (a cudaStream_t, NULL = legacy default stream).  Device memory is
 * not allocated here: attach a workspace with pswf_plan_set_workspace, or the
 * first pswf_set_points allocates one (cudaMalloc) that the plan owns. */
int pswf_plan_create(const double box[3], int64_t n_max, int K, const int* p,
                     const pswf_opts* opts, void* stream, pswf_plan* out);

/* A single structure in a general (triclinic) periodic cell.
 * cell: host [9], the lattice vectors a_0, a_1, a_2 as rows (Angstrom); the
 * positions are Cartesian (any real value: wrapped through the fractional
 * coordinates).  The grid is uniform in the fractional coordinates (M_d
 * points along a_d), the window and its deconvolution act per grid direction
 * and the modes are k = 2 pi H^-1 m (Methods, with the box replaced by the
 * cell: Eq. (Fourier) sums over the reciprocal lattice); grid, P and c_w are
 * chosen for the edge lengths |a_d|.  Forces are Cartesian.  Otherwise as
 * pswf_plan_create (pswf_backward and pswf_stress included: dL/dr and the
 * virial tensor are Cartesian too); an orthorhombic cell gives the box plan.
 * Returns PSWF_EINVAL for non-finite or (nearly) coplanar vectors. */
int pswf_plan_create_cell(const double cell[9], int64_t n_max, int K, const int* p, const pswf_opts* opts,
                          void* stream, pswf_plan* out);

/* Fills *out; synchronous, host only. */
int pswf_plan_info(pswf_plan plan, pswf_info* out);

/* Attaches caller-owned device memory of at least info.workspace_bytes bytes,
 * 256-byte aligned, which must outlive the plan's use of it.  Uploads the
 * plan's tables into it (synchronous copies). */
int pswf_plan_set_workspace(pswf_plan plan, void* workspace, int64_t bytes);

/* Changes the stream later calls enqueue on. */
int pswf_plan_set_stream(pswf_plan plan, void* stream);

/* Sets the input of step (i) of "Accelerating atom-grid spreading with
 * PSWFs" (the atoms whose latent charges are spread onto the grid): bins and
 * sorts the atoms by grid tile (new positions and/or charges), computes each
 * atom's stencil start and window offsets (Eq. for W_pswf: P points per
 * dimension around r / h), the per-channel charge sums used by the
 * zero-frequency and self terms, and the spread's per-tile fixed-point units.
 * pos: device [n][3] float (pos_dtype 0) or double (pos_dtype 1), any real
 *   values (wrapped into the box);
 * q:   device [K][n] real latent charges.
 * Both are read during this call's kernels only (stream-ordered).
 * n must be 0..n_max.  NaN/Inf positions are reported by the next
 * synchronising call as PSWF_ENONFINITE (those atoms are binned at 0). */
int pswf_set_points(pswf_plan plan, int64_t n, const void* pos, int pos_dtype, const void* q);

/* Forward evaluation of the points last set (asynchronous).
 * energy: device double [K + 1] (may be NULL): E_c per channel (Eq. Fourier,
 *   reciprocal sum plus zero-frequency term), total at [K];
 * phi:    device real [K][n] (may be NULL): phi_i^(c) = dE/dq_i^(c);
 * forces: device real [n][3] (may be NULL): F_i = -dE/dr_i summed over channels.
 * When the plan has PSWF_FLAG_BACKWARD the grid potential is kept for
 * pswf_backward. */
int pswf_execute(pswf_plan plan, double* energy, void* phi, void* forces);

/* ---- batches of structures ---------------------------------------------
 * A batch plan evaluates up to b_max independent structures per call, each
 * with its own orthorhombic box and atoms, all on one grid size (the serving
 * and training workloads: many small systems).  Per structure the result is
 * the same computation as a single-structure plan with the same grid, c_w
 * and P; the paper evaluates one structure at a time and has no counterpart
 * for the batching itself.
 *
 * pswf_batch_plan_create: box_max host [3] is the largest box edge per axis
 * any structure may have; the grid (opts->grid or the planner's choice),
 * eta, c_w and P are chosen at box_max, so every smaller box is on a finer
 * grid (smaller eta: the same window stays alias-free).  pset host [npset]
 * lists the exponents channels may use (multiplier tables are built for
 * these only).  n_max is the total atom capacity of one call.  The energy of
 * pswf_execute becomes device double [b_max][K + 1]; phi and forces keep the
 * [K][n] and [n][3] layouts over the concatenated atoms but must hold n_max
 * entries (rows) each; pswf_self_energy fills host double [b_max][K];
 * pswf_backward takes g_energy as device double [b_max][K].
 * pswf_set_points, pswf_compute_host and pswf_self_energy_noalloc reject
 * batch plans (PSWF_EINVAL). */
int pswf_batch_plan_create(const double box_max[3], int b_max, int64_t n_max, int K, const int* pset, int npset,
                           const pswf_opts* opts, void* stream, pswf_plan* out);

/* Sets the structures of the next pswf_execute.  b (0..b_max) structures;
 * boxes host double [b][3] (each edge <= box_max); ps host int [b][K]
 * exponents (from the plan's pset); offsets host int64 [b + 1], offsets[0] =
 * 0, non-decreasing: structure s owns atoms offsets[s] .. offsets[s+1] - 1 of
 * pos (device [n][3], float or double) and of q (device real [K][n]), n =
 * offsets[b] <= n_max.  Slots b..b_max-1 are empty (zero energy).  Later
 * launches cover only the smallest planned slot count >= b (1, 2, 4, ...,
 * b_max; one cuFFT plan pair each), so a small batch costs little.  The box
 * tables are computed on the host into a pinned buffer owned by the plan and
 * copied on the plan's stream; a later call first waits for that copy. */
int pswf_batch_set_points(pswf_plan plan, int b, const double* boxes, const int* ps, const int64_t* offsets,
                          const void* pos, int pos_dtype, const void* q);

/* Vector-Jacobian product of the last pswf_execute (asynchronous; needs
 * PSWF_FLAG_BACKWARD and the same points): the derivatives the paper obtains
 * by automatic differentiation of the long-range energy (forces, and the
 * gradients that train the latent charges; Fig. 1 caption), written here as
 * the exact adjoint of the discrete spread / transform / multiplier / gather
 * operator: one more spread (of g_phi W and q g_F . grad W), transform pair
 * and gather (with the Hessian of W for the force term).  Upstream gradients, each may be
 * NULL (= zero): g_energy device double [K] (d loss / d E_c), g_phi device
 * real [K][n], g_forces device real [n][3].  Outputs (may be NULL):
 * grad_q device real [K][n], grad_pos device real [n][3]. */
int pswf_backward(pswf_plan plan, const double* g_energy, const void* g_phi,
                  const void* g_forces, void* grad_q, void* grad_pos);

/* Self energies E_self^(p) ("Implementation details") of the points last set,
 * host double [K].  Synchronises the stream. */
int pswf_self_energy(pswf_plan plan, double* out);

/* Self energies like pswf_self_energy, for callers that must not allocate
 * device memory while they run -- for example a plug-in inside a molecular
 * dynamics engine that owns every GPU buffer and forbids allocation once the
 * simulation loop has started, or a process that has handed all free device
 * memory to its own pool.  The paper has no counterpart: it is a different
 * way to run the same per-channel reduction.
 *   plan:   read only for its host-side constants (the self-energy
 *           coefficients); its workspace, stream and points are not used;
 *   n, q:   device real [K][n] latent charges (plan precision), n <= n_max;
 *   out:    device double [K]: E_self^(p) per channel (caller-owned);
 *           q and out live on the plan's device, which must be the current
 *           device at the call (PSWF_EINVAL otherwise);
 *   stream: cudaStream_t the work is enqueued on (asynchronous).
 * Allocates nothing: the FP64 partial sums live in a 152,576-byte array of
 * static device memory inside this library, which every GPU that loads the
 * library holds until the process exits.  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress, with that device
 * current); make that first call before any stream capture.  Every call on a
 * device shares the one array: calls whose work overlaps on the GPU (other
 * streams, other threads) race and give wrong results; serialise them.  Each
 * call writes every scratch entry before reading it, so nothing has to be
 * cleared.  Returns PSWF_EINVAL for n outside 0..n_max or more than 64
 * channels (the array's limit). */
int pswf_self_energy_noalloc(pswf_plan plan, int64_t n, const void* q, double* out, void* stream);

/* Diagonal virial of the last pswf_execute (plan created with
 * PSWF_FLAG_VIRIAL), device double [B][K][3] (B = 1 for single structures):
 * W_cd = -L_d dE_c/dL_d at fixed fractional coordinates (for a box; in a
 * general cell the Cartesian diagonal of pswf_stress), E_c the channel
 * energy of pswf_execute (reciprocal sum and zero-frequency term; the
 * self-energy does not depend on the box).  The grid density and the window
 * transform are invariant under that scaling, so W_cd = E_c + sum_m e_m
 * (d ln Phi-hat_p / d ln k) k_d^2 / k^2 over the band modes m with energy
 * terms e_m (Eq. (Fourier), Eq. (PhiH)).  The stress of the cell is -W / V.
 * Asynchronous on the plan's stream. */
int pswf_virial(pswf_plan plan, double* virial);

/* Virial tensor of the last pswf_execute (plan created with
 * PSWF_FLAG_VIRIAL), device double [B][K][6] as (xx, yy, zz, xy, xz, yz):
 * W_ab = -dE_c / d epsilon_ab under the symmetric strain r -> (1 + epsilon) r
 * of the cell vectors and the atoms together (fixed fractional
 * coordinates; any cell).  The grid density and the window transform are
 * strain-invariant and k -> (1 - epsilon) k, V -> (1 + tr epsilon) V, so
 * W_ab = E_c delta_ab + sum_m e_m (d ln Phi-hat_p / d ln k) k_a k_b / k^2
 * (stress for constant-pressure runs; the paper has no stress).  Stress = -W / V.
 * Asynchronous on the plan's stream. */
int pswf_stress(pswf_plan plan, double* virial);

/* Real-space complement (Methods, "Implementation details": the
 * pair term that completes Eq. (Fourier); G_p taken as 1 beyond r_c):
 *   E_c = 1/2 sum_{i != j, |r_ij| < r_c} q_i^c q_j^c (1 - G_p(r_ij)) / r_ij^p
 * with G_p of Eq. G1, G6, G (the planner's piecewise polynomial in r / r_c),
 * its potentials phi_i^c = dE_c / dq_i^c and forces.  With the reciprocal part
 * of pswf_execute and the self energies (pswf_self_energy) it gives the
 * complete 1/r^p lattice sum: E = E_recip + E_real - E_self, phi and F the
 * sums likewise (phi also takes -2 s_p q_i from the self energy).  Plans
 * created with PSWF_FLAG_REAL_SPACE (single structures in a box or a general
 * cell, K <= 16).  When every height of the cell across a pair of faces is
 * at least 3 r_c a cell list is used (>= 3 list cells per lattice vector,
 * each at least r_c high, so each pair is found once, in its nearest
 * image); otherwise every pair of atoms is summed over the images n H that
 * can come closer than r_c (minimum image for r_c <= L/2, more images
 * beyond), for at most 16384 atoms.  Inputs as
 * pswf_set_points (positions any real value, wrapped; q real [K][n] in the
 * plan's precision); it does not touch the sorted atoms of pswf_set_points.
 * energy: device double [K + 1] (per channel, total), written; phi: real
 * [K][n], forces: real [n][3], written, either may be NULL.  Asynchronous on
 * the plan's stream; pswf_sync reports non-finite positions
 * (PSWF_ENONFINITE) and a list cell holding more than 2048 atoms
 * (PSWF_ECELL: such a cell's pairs are left out; no liquid or solid comes
 * near that density).  Errors: PSWF_ESTATE without PSWF_FLAG_REAL_SPACE;
 * PSWF_EINVAL for a null energy, n outside 0..n_max, missing pos / q or a
 * bad pos_dtype (pswf_plan creation with the flag already returned
 * PSWF_EINVAL for a batch, K > 16, a direct sum over more than 16384
 * atoms or r_c needing more than 4096 images); PSWF_ECUDA if a launch
 * fails. */
int pswf_real_space(pswf_plan plan, int64_t n, const void* pos, int pos_dtype, const void* q, double* energy,
                    void* phi, void* forces);

/* Vector-Jacobian product of pswf_real_space's outputs (asynchronous; needs
 * a preceding pswf_real_space on the same atoms, whose cell list it reuses):
 * the gradients of L = sum_c g_energy_c E_c + sum g_phi * phi + sum g_forces
 * . F through the pair term of "Implementation details", the derivatives the
 * paper takes by automatic differentiation of the complete energy (Fig. 1
 * caption), here per atom over its neighbours with G_p and its first two
 * derivatives (the force term needs f_p'').
 * pos, pos_dtype, q: the same inputs as that pswf_real_space call;
 * upstream (each may be NULL = zero): g_energy device double [K], g_phi
 * device real [K][n], g_forces device real [n][3];
 * outputs (may be NULL, written, not accumulated): grad_q device real [K][n],
 * grad_pos device real [n][3].
 * PSWF_ESTATE without the preceding call (or for another atom count). */
int pswf_real_space_backward(pswf_plan plan, int64_t n, const void* pos, int pos_dtype, const void* q,
                             const double* g_energy, const void* g_phi, const void* g_forces, void* grad_q,
                             void* grad_pos);

/* Waits for the plan's stream and returns the first device-side status
 * raised since the last call (e.g. PSWF_ENONFINITE), clearing it. */
int pswf_sync(pswf_plan plan);

/* pswf_sync with a limit: polls the stream and returns PSWF_ETIMEOUT if its
 * work is still running after timeout_ms milliseconds (the work continues;
 * call again to wait further); timeout_ms < 0 waits without limit.  The
 * paper has no counterpart (a host-side bounded wait). */
int pswf_sync_for(pswf_plan plan, double timeout_ms);

/* End-to-end evaluation from host memory (synchronising): copies positions
 * (host double [n][3]) and charges (host double [K][n]) to the device,
 * runs set_points + execute, and copies back energy (host double [K + 1]),
 * phi (host double [K][n], may be NULL) and forces (host double [n][3], may
 * be NULL).  Page-locked caller arrays (cudaHostAlloc, cudaMallocHost or
 * cudaHostRegister) are copied directly: positions and charges in (FP32
 * plans round the charges on the device), potentials and forces out (FP32
 * results widened to double on the device first, so the copy out is K n 8 +
 * 24 n bytes).  Pageable arrays go through pinned staging buffers owned by
 * the plan, filled and drained by host threads in chunks overlapped with the
 * copies (charges rounded to the plan's precision there).  Synchronises the
 * plan's stream. */
int pswf_compute_host(pswf_plan plan, int64_t n, const double* pos, const double* q,
                      double* energy, double* phi, double* forces);

/* pswf_compute_host with charges, potentials and forces in the plan's
 * precision (float for FP32 plans, double for FP64 plans): q host real
 * [K][n], phi host real [K][n] (may be NULL), forces host real [n][3] (may
 * be NULL); positions host double [n][3] and energy host double [K + 1] as
 * above.  Page-locked arrays are copied as they are, with no conversion on
 * either side (an FP32 plan moves 24 n + 4 K n bytes in and 4 K n + 12 n
 * out); pageable ones go through the plan's pinned staging buffers.  Same
 * errors as pswf_compute_host.  The paper has no counterpart (host
 * transfers). */
int pswf_compute_host_real(pswf_plan plan, int64_t n, const double* pos, const void* q,
                           double* energy, void* phi, void* forces);

/* Releases everything the plan owns (not a caller-attached workspace).
 * Freeing device memory waits for all outstanding work on the device, so a
 * plan destroyed while a server runs stalls the server's streams until
 * then: destroy plans outside latency-critical windows. */
void pswf_plan_destroy(pswf_plan plan);

/* Human-readable name of a status code (static string). */
const char* pswf_strerror(int status);

/* Copies the plan's last error message into buf (NUL-terminated). */
int pswf_plan_last_error(pswf_plan plan, char* buf, int len);

/* ---- request server (continuous batching; not part of the paper) ------
 * Serves independent structures (each: n atoms, an orthorhombic box, K
 * channels with exponents from pset) over batch plans.  Every structure is
 * routed to the smallest bucket whose cubic grid covers its largest box edge
 * at spacing h_max and whose batch holds its atoms; its result is what a
 * batch plan of that bucket gives for it alone.  Each bucket owns `inflight`
 * batch contexts (plan, stream, device buffers, pinned staging) allocated at
 * creation, so device memory is fixed; a scheduler thread hands the
 * bucket's oldest requests to every free context (up to b_max structures and
 * n_max atoms), and with use_graphs the context's kernels run as one
 * captured CUDA graph per batch.  Submit and wait are thread-safe. */
#define PSWF_MAX_BUCKETS 16
typedef struct pswf_server_s* pswf_server;

typedef struct {
  double r_c, tol, c;             /* method parameters as in pswf_opts (c 0 -> log(3 / tol)) */
  double h_max;                   /* largest grid spacing (A); 0 -> 0.5 pi r_c / c (eta = 0.5) */
  int K;                          /* channels per structure */
  int npset;                      /* number of exponents in pset */
  int pset[6];                    /* exponents channels may use */
  int nbucket;                    /* buckets, 1..PSWF_MAX_BUCKETS */
  int grid[PSWF_MAX_BUCKETS];     /* cubic grid size per bucket, strictly ascending */
  int b_max[PSWF_MAX_BUCKETS];    /* structures per batch of each bucket */
  int64_t n_max[PSWF_MAX_BUCKETS];/* atoms per batch of each bucket */
  int inflight;                   /* batch contexts per bucket (default 2) */
  int precision;                  /* 0: FP32 path, 1: FP64 */
  int use_graphs;                 /* 1 (default): replay one captured CUDA graph per batch */
  int P;                          /* stencil width; 0 -> planner */
} pswf_server_opts;

/* Defaults: tol 1e-5, inflight 2, use_graphs 1, everything else 0. */
void pswf_server_opts_default(pswf_server_opts* o);

/* Creates the buckets' plans and buffers on the current device and starts
 * the scheduler thread.  PSWF_EINVAL for bad options, PSWF_ENOMEM if the
 * contexts do not fit. */
int pswf_server_create(const pswf_server_opts* opts, pswf_server* out);

/* Bucket a structure of n atoms with edges box (host [3]) would use: returns
 * its index (>= 0) and, if info != NULL, fills it with that bucket's plan
 * parameters (grid, P, c, c_w, ...); PSWF_EINVAL if no bucket holds it. */
int pswf_server_route(pswf_server srv, int64_t n, const double box[3], pswf_info* info);

/* Queues one structure: box host [3], ps host [K], pos host double [n][3],
 * q host double [K][n] (copied before returning; FP32 plans round q).
 * *ticket identifies it for pswf_server_wait.  PSWF_EINVAL if no bucket
 * holds it or an exponent is not in pset; a failed server returns its
 * status. */
int pswf_server_submit(pswf_server srv, int64_t n, const double box[3], const int* ps, const double* pos,
                       const double* q, int64_t* ticket);

/* Blocks until the structure is done and copies its results: energy host
 * double [K + 1] (per channel, total last), phi host double [K][n] and forces
 * host double [n][3] (either may be NULL); latency_ms (may be NULL) = time
 * from submit to the completion of its batch.  The ticket is released. */
int pswf_server_wait(pswf_server srv, int64_t ticket, double* energy, double* phi, double* forces,
                     double* latency_ms);

/* pswf_server_wait with a limit: returns PSWF_ETIMEOUT if the structure is
 * not done within timeout_ms milliseconds (the ticket stays valid and can be
 * waited for again); timeout_ms < 0 waits without limit.  The paper has no
 * counterpart (host-side serving). */
int pswf_server_wait_for(pswf_server srv, int64_t ticket, double timeout_ms, double* energy, double* phi,
                         double* forces, double* latency_ms);

/* pause != 0: the scheduler starts no new batch (batches in flight finish
 * and are collected; submissions queue); pause = 0 resumes.  For draining a
 * server before a reconfiguration, or holding requests back. */
int pswf_server_pause(pswf_server srv, int pause);

/* Submits count structures in one call (as count pswf_server_submit calls,
 * in order): n host int64 [count] atoms per structure, boxes host double
 * [count][3], ps host int [count][K], pos host array [count] of pointers to
 * each structure's positions (double [n_i][3]), q host array [count] of
 * pointers to its charges (double [K][n_i]); tickets host int64 [count]
 * receives the tickets.  flags 0: the inputs are copied before the call
 * returns; PSWF_SUBMIT_BORROW: they are only referenced, read when the
 * structure's batch is staged, and the caller keeps them valid and
 * unchanged until the structure has been waited for.  On an error the
 * structures before the failing one stay submitted (their tickets are
 * written); PSWF_EINVAL for unknown flags.  For clients that hand over many
 * structures at once. */
#define PSWF_SUBMIT_BORROW 1
int pswf_server_submit_many(pswf_server srv, int64_t count, const int64_t* n, const double* boxes, const int* ps,
                            const double* const* pos, const double* const* q, int64_t* tickets, int flags);

/* Waits for count tickets (as pswf_server_wait, in order) and writes each
 * structure's results: energies host double [count][K + 1], phi host double
 * with structure i's [K][n_i] at phi + K offsets[i] (may be NULL), forces
 * host double [offsets[count]][3] (may be NULL), latency_ms host double
 * [count] (may be NULL); offsets host int64 [count + 1], the running sums of
 * the structures' atom counts.  Every ticket is waited for and released;
 * returns the first error. */
int pswf_server_wait_many(pswf_server srv, int64_t count, const int64_t* tickets, const int64_t* offsets,
                          double* energies, double* phi, double* forces, double* latency_ms);

/* Counters since creation (any may be NULL); returns the server's failure
 * status (0 if healthy). */
int pswf_server_stats(pswf_server srv, int64_t* batches, int64_t* requests, int64_t* atoms);

/* Message of the last server failure. */
int pswf_server_last_error(pswf_server srv, char* buf, int len);

/* Stops the scheduler, waits for batches in flight and frees everything;
 * tickets not yet waited for are dropped. */
void pswf_server_destroy(pswf_server srv);

/* ---- measurement support (not part of the paper's method) -------------- */
#define PSWF_NSTAGE 11
/* Stage indices for pswf_profile_read. */
#define PSWF_STAGE_SET_POINTS 0   /* binning, sort, charge sums */
#define PSWF_STAGE_SPREAD 1       /* step (i) */
#define PSWF_STAGE_FFT_FWD 2      /* step (ii), cuFFT */
#define PSWF_STAGE_MULTIPLY 3     /* steps (iii)-(iv) and the energy reduction */
#define PSWF_STAGE_FFT_INV 4      /* inverse transform, cuFFT */
#define PSWF_STAGE_INTERP 5       /* gather of potentials and forces */
#define PSWF_STAGE_BACKWARD 6     /* pswf_backward */
#define PSWF_STAGE_OTHER 7
#define PSWF_STAGE_REAL_SPACE 8   /* pswf_real_space (cell list and pairs) */
#define PSWF_STAGE_H2D 9          /* pswf_compute_host: call entry to the last input copy's end
                                     (host staging of the first chunk included) */
#define PSWF_STAGE_D2H 10         /* pswf_compute_host: end of the evaluation to the last output
                                     copy's end */

/* enable != 0: later calls record a CUDA event pair around each stage on the
 * plan's stream (costs one event record per stage boundary). */
int pswf_profile_enable(pswf_plan plan, int enable);

/* Synchronises the stream and returns, per stage, the summed event time in
 * milliseconds (host double [PSWF_NSTAGE], may be NULL) and the number of
 * this library's own kernels launched (host int64 [PSWF_NSTAGE], may be NULL;
 * cuFFT's kernels and memsets are not counted) since the last read; then
 * resets both. */
int pswf_profile_read(pswf_plan plan, double* stage_ms, int64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* PSWF_LR_H */
