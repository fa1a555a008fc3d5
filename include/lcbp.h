/*
 * lcbp.h -- C ABI of liblcbp.so, the GB300 (sm_103a) implementation of the
 * coupled hybrid lattice-Boltzmann / Beris-Edwards step of
 * Henrich, Marenduzzo, Stratford, Cates, "Domain growth in cholesteric blue
 * phases: hybrid lattice Boltzmann simulations" (arXiv:0901.3293).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every call returns an int status: LCBP_OK (0) or a negative LCBP_E* code.
 *   lcbp_strerror() names a code; lcbp_last_error() returns a thread-local
 *   message describing the last failure of the calling thread.  No call
 *   aborts the process, traps the GPU or leaves a kernel waiting forever.
 * - Lattice sites are indexed s = (z * ny + y) * nx + x (x fastest), periodic
 *   in all three directions.  Fields cross the boundary in structure-of-arrays
 *   layout [component][z][y][x]:
 *     Q : 5 components [xx, xy, xz, yy, yz]; Q_zz = -Q_xx - Q_yy (Q is
 *         symmetric and traceless, Sec. 2.1 and the 5-value storage of Sec. 2.2).
 *     u : 3 components [ux, uy, uz];  rho : 1 component.
 *     f : 15 D3Q15 populations (Sec. 2.2 Eq. latvects) in the order
 *         0 rest; 1..6 = +x, -x, +y, -y, +z, -z;
 *         7..14 = (+1,+1,+1), (+1,+1,-1), (+1,-1,+1), (+1,-1,-1),
 *                 (-1,+1,+1), (-1,+1,-1), (-1,-1,+1), (-1,-1,-1).
 * - Buffer arguments (const void *src / void *dst) may be host memory
 *   (pageable or pinned) or device memory of the current device (unified
 *   addressing decides); `dtype` (LCBP_F32 / LCBP_F64) is their element type,
 *   converted to and from the lattice's state type.  Reads are synchronous:
 *   the data is in `dst` when the call returns.  The caller owns every buffer
 *   it passes; the library keeps no pointer to it after returning.
 * - Ownership of device memory: lcbp_create allocates the lattice's state and
 *   scratch with cudaMalloc and frees it in lcbp_destroy.
 *   lcbp_create_on_buffers instead works inside a caller-owned device
 *   workspace (e.g. a PyTorch tensor) on a caller-owned stream; the library
 *   never frees either, and the caller must keep both alive until
 *   lcbp_destroy.  Diagnostics use a few kilobytes of library-allocated
 *   device memory in both cases.
 * - Work is enqueued on the lattice's stream.  lcbp_step returns once the
 *   steps are enqueued; reads and diagnostics synchronise the stream.
 * - Lattice units throughout: dx = dt = 1.
 * - Internally the populations are stored as deviations f_i - w_i from the
 *   rest-state weights w = (8/15, 1/30, ..., 1/30) and the density as rho - 1,
 *   which keeps FP32 state accurate (mass is conserved to the rounding of
 *   O(1e-3) numbers).  The boundary always exchanges full f and rho.
 */
#ifndef LCBP_H
#define LCBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define LCBP_API __attribute__((visibility("default")))
#else
#define LCBP_API
#endif

#define LCBP_VERSION 1

/* status codes */
#define LCBP_OK 0
#define LCBP_EINVAL (-1)      /* bad argument (null handle, size, dtype, kind ...) */
#define LCBP_ENOMEM (-2)      /* device or host allocation failed / workspace too small */
#define LCBP_ECUDA (-3)       /* a CUDA runtime call or kernel launch failed */
#define LCBP_ENONFINITE (-4)  /* a diagnostic found NaN or Inf in the state */
#define LCBP_ETIMEOUT (-5)    /* a bounded device-side wait gave up */
#define LCBP_ESTATE (-6)      /* call out of order (e.g. stepping before init) */
#define LCBP_EIO (-7)         /* checkpoint file could not be read or written */

/* element types of state and of caller buffers */
#define LCBP_F32 0
#define LCBP_F64 1

/* initial order-parameter kinds (lcbp_init_q) */
#define LCBP_BPII 0              /* simple-cubic blue phase II seed (O2 structure) */
#define LCBP_CHOL_X 1            /* cholesteric helix, axis x: n = (0, cos q0x, sin q0x) */
#define LCBP_CHOL_Y 2            /* axis y: n = (sin q0y, 0, cos q0y) */
#define LCBP_CHOL_Z 3            /* axis z: n = (cos q0z, sin q0z, 0) */
#define LCBP_ISO_NOISE 4         /* isotropic Q = 0 plus noise */
#define LCBP_SLAB_BPII_IN_CHOL 5 /* BPII for z < region[0], x-helix elsewhere */
#define LCBP_SLAB_BPII_IN_ISO 6  /* BPII for z < region[0], isotropic (noise only) elsewhere (Sec. 3, Fig. 3) */
#define LCBP_SLAB_BPII_IN_CHOL_Z 7 /* BPII for z < region[0], z-helix (axis normal to the wall) elsewhere (Sec. 3) */

/* order of the two sub-updates within one step (Sec. 2.2: "sequentially updated") */
#define LCBP_JACOBI 0       /* LB and Q both read the step-n fields (default) */
#define LCBP_GAUSS_SEIDEL 1 /* LB first, then Q advanced with u^{n+1} */

/* kernel selection (lcbp_set_path) */
#define LCBP_PATH_AUTO 0    /* fast z-marching TMA kernels where they apply, else generic */
#define LCBP_PATH_GENERIC 1 /* always the generic one-thread-per-site kernels */
#define LCBP_PATH_FAST1 2   /* as AUTO, fast kernels pinned to one site per thread */
#define LCBP_PATH_FAST2 3   /* as AUTO, fast kernels pinned to two sites per thread (FP32 only) */

typedef struct lcbp_lattice lcbp_lattice;

/* Name of a status code (static string). */
LCBP_API const char *lcbp_strerror(int code);
/* Message of the calling thread's last failure ("" if none). */
LCBP_API const char *lcbp_last_error(void);
/* LCBP_VERSION of the loaded library. */
LCBP_API int lcbp_version(void);

/*
 * Create a periodic nx * ny * nz lattice (each >= 1) with state type
 * LCBP_F32 or LCBP_F64 on the current CUDA device, allocating its memory and
 * a non-blocking stream.  Parameters start at the defaults A0 = 0.01,
 * gamma = 3.1, K = 0.01, q0 = 2 pi / 16, tau_f = 2, xi = 0.7, Gamma = 0.3,
 * flow on, Jacobi coupling; Q = 0 and f = 0 until initialised.
 * Errors: LCBP_EINVAL (sizes < 1, more than 2^31 sites, bad dtype, out == NULL),
 * LCBP_ENOMEM, LCBP_ECUDA.
 */
LCBP_API int lcbp_create(int nx, int ny, int nz, int state_dtype, lcbp_lattice **out);

/* Bytes of device workspace lcbp_create_on_buffers needs for this lattice. */
LCBP_API size_t lcbp_workspace_bytes(int nx, int ny, int nz, int state_dtype);

/*
 * As lcbp_create, but the state and scratch live in the caller's device
 * buffer `workspace` (at least lcbp_workspace_bytes, 256-byte aligned) and
 * work goes to the caller's stream (a cudaStream_t passed as void*, NULL for
 * the legacy default stream).  Errors: as lcbp_create; LCBP_ENOMEM if
 * workspace_bytes is too small, LCBP_EINVAL if workspace is misaligned.
 */
LCBP_API int lcbp_create_on_buffers(int nx, int ny, int nz, int state_dtype, void *workspace,
                           size_t workspace_bytes, void *stream, lcbp_lattice **out);

/* Release everything the library allocated for h (NULL is accepted). */
LCBP_API int lcbp_destroy(lcbp_lattice *h);

/* nx, ny, nz, state dtype and number of completed steps. */
LCBP_API int lcbp_get_info(const lcbp_lattice *h, int dims[3], int *state_dtype, long long *step);

/*
 * Landau-de Gennes parameters of Sec. 2.1 Eq. (free_energy): A0, gamma, the
 * one-constant elastic constant K (= L1 of the kappa definition) and q0 = 2 pi / pitch.
 * The gradient energy is the one-constant form
 *   (K/2)|grad Q|^2 + 2 K q0 Q:(eps grad Q) + 2 K q0^2 |Q|^2,
 * i.e. the printed chiral square plus (K/2)(d_b Q_ab)^2 up to a divergence.
 * Errors: LCBP_EINVAL (A0 <= 0, gamma <= 0, K < 0, non-finite values).
 */
LCBP_API int lcbp_set_ldg(lcbp_lattice *h, double A0, double gamma, double K, double q0);

/*
 * Same, from the reduced chirality kappa and temperature tau of Sec. 2.1:
 * gamma = 27 / (9 + tau), K = kappa^2 A0 gamma / (108 q0^2).
 * Errors: LCBP_EINVAL (tau <= -9, q0 == 0, kappa < 0).
 */
LCBP_API int lcbp_set_ldg_kappa_tau(lcbp_lattice *h, double A0, double q0, double kappa, double tau);

/*
 * Kinetic parameters: LB relaxation time tau_f (viscosity eta = rho tau_f / 3,
 * Sec. 2.2 Eq. eq4), reference density rho0 of the fluid (the density of the
 * initial equilibrium, Sec. 2.2 Eq. feq; lcbp_init_f_equilibrium uses it when
 * given 0; default 1), flow-aligning parameter xi (Sec. 2.1 Eq. mat_der),
 * rotational diffusion constant Gamma (Eq. Qevolution), flow_on (0 imposes
 * u = 0 and skips the LB update, Sec. 2.1), coupling LCBP_JACOBI or
 * LCBP_GAUSS_SEIDEL.  Errors: LCBP_EINVAL (tau_f <= 0, rho0 <= 0, Gamma < 0,
 * bad coupling).
 */
LCBP_API int lcbp_set_flow(lcbp_lattice *h, double tau_f, double rho0, double xi, double Gamma, int flow_on,
                           int coupling);

/*
 * Elastic energy variant (Sec. 2.1, Eq. free_energy).  The printed gradient
 * energy is the chiral square (K/2)(eps dQ + 2 q0 Q)^2; on a periodic domain
 * it equals the one-constant energy (K/2)|grad Q|^2 + 2 K q0 Q:(eps grad Q) +
 * 2 K q0^2 |Q|^2 minus (K/2)(d_b Q_ab)^2.  By default (use_l2 = 0) the library
 * uses the one-constant energy; with use_l2 != 0 the energy gains
 * -((K - L2)/2) sum_x |div Q|^2, div_a = sum_b D0_b Q_ab (central differences),
 * and H its exact lattice gradient: L2 = 0 is the energy exactly as printed,
 * L2 = K the default.  Lattices with L2 != K run the generic kernels.
 * Errors: LCBP_EINVAL (non-finite L2; walls set).
 */
LCBP_API int lcbp_set_l2(lcbp_lattice *h, int use_l2, double L2);

/*
 * Solid walls in z (not in the paper, whose slab is periodic; an extension).
 * With walls_z != 0 the lattice has walls half a spacing below z = 0 and above
 * z = Nz-1, while x and y stay periodic:
 *  - LB: half-way bounce-back (no slip): a population that would arrive from
 *    beyond a wall is the reflected one of the same site;
 *  - Q: strong anchoring, the ghost planes z = -1 and z = Nz hold Q = q_wall5
 *    (q5 order [xx, xy, xz, yy, yz]; NULL = 0) in every stencil;
 *  - u: no slip, ghost u = -u of the adjacent plane (velocity gradient,
 *    advection);
 *  - tau and H vanish on the ghost planes (body force).
 * The free energy then counts every bond with at least one end on the
 * lattice, so H stays its exact gradient.  Walled lattices run the fast
 * kernels (one site per thread) where the fast path applies, else the generic
 * ones; the surrogate refuses them.  walls_z = 0 restores periodic z.  Every
 * call re-records the captured step (q_wall is a launch argument).
 * Errors: LCBP_EINVAL (non-finite q_wall; L2 set).
 */
LCBP_API int lcbp_set_walls(lcbp_lattice *h, int walls_z, const double *q_wall5);

/*
 * Fill Q with an analytic initial state on the device (kinds above):
 * BPII:  Q_xx = A[cos 2q0z - cos 2q0y], Q_yy = A[cos 2q0x - cos 2q0z],
 *        Q_xy = A sin 2q0z, Q_xz = A sin 2q0y, Q_yz = A sin 2q0x (A = amplitude);
 * CHOL_*: Q = S (n n - I/3), S = amplitude;  ISO_NOISE: Q = 0;
 * SLAB_BPII_IN_CHOL: BPII (A = amplitude) for z < region[0], elsewhere the
 *   x-helix with S = 1/4 + 3/4 sqrt(1 - 8 / (3 gamma)) (bulk equilibrium order);
 * SLAB_BPII_IN_CHOL_Z: the same with the z-helix (axis normal to the wall);
 * SLAB_BPII_IN_ISO: BPII for z < region[0], Q = 0 elsewhere (Sec. 3, the
 *   seed growing into the isotropic phase).
 * Then add U[-noise, noise) to each of the five components, the k-th output
 * (k = 5 * site + component) of SplitMix64 seeded with `seed`, mapped to
 * (z >> 11) * 2^-53.  region may be NULL except for the SLAB_* kinds.
 * Errors: LCBP_EINVAL (unknown kind, missing region, noise < 0).
 */
LCBP_API int lcbp_init_q(lcbp_lattice *h, int kind, double amplitude, double noise, uint64_t seed,
                const int *region);

/* Upload Q: q5 holds 5 * N values in the layout above.  A field holding any
 * NaN or Inf is refused and Q is left unchanged.  Errors: LCBP_EINVAL,
 * LCBP_ENONFINITE. */
LCBP_API int lcbp_set_q(lcbp_lattice *h, const void *q5, int dtype);

/*
 * Set f = f^eq(rho0, u, sigma_LC(Q)) at every site (Sec. 2.2 Eq. feq, coeff,
 * without the forcing term), with u from u3 (3 * N values) or u = 0 if u3 is
 * NULL, and sigma_LC from the current Q; rho0 = 0 takes the reference density
 * of lcbp_set_flow.  Errors: LCBP_EINVAL (rho0 < 0).
 */
LCBP_API int lcbp_init_f_equilibrium(lcbp_lattice *h, double rho0, const void *u3, int dtype);

/* Upload the 15 * N populations.  Populations holding any NaN or Inf are
 * refused and f is left unchanged.  Errors: LCBP_EINVAL, LCBP_ENONFINITE. */
LCBP_API int lcbp_set_f(lcbp_lattice *h, const void *f15, int dtype);

/*
 * Optional external body force (3 * N values) added to the LC body force b of
 * Sec. 2.2 Eq. (eq7a) in the LB forcing; NULL removes it.
 */
LCBP_API int lcbp_set_body_force(lcbp_lattice *h, const void *b3, int dtype);

/*
 * Advance nsteps >= 0 coupled steps (Sec. 2.2): molecular field H, LC stress
 * sigma_LC and tau, body force b = D0_b tau_ab - H_gn D0_a Q_gn (Eq. spurious),
 * predictor-corrector D3Q15 LB with BGK + forcing (Eq. eq2, eq4), and the Heun
 * predictor-corrector for Q with central differences (Eq. Qevolution,
 * mat_der).  Returns once the work is enqueued (CUDA-graph replay).
 * Errors: LCBP_ESTATE (f never initialised while flow is on), LCBP_ECUDA.
 */
LCBP_API int lcbp_step(lcbp_lattice *h, int nsteps);

/*
 * Advance nsteps >= 1 steps exactly as lcbp_step does, but launched one kernel
 * at a time with a CUDA event between kernels, and return in kernel_ms the
 * mean device time of each kernel of one step (milliseconds).  *nkernels is
 * set to the number of kernels per step: 2 on the fast path (qside: H, sigma,
 * tau, b and the Heun predictor; lbq: LB predictor-corrector and the Heun
 * corrector); on the generic path 3 with flow on and Jacobi coupling
 * (field: H/sigma/tau; force_predict: b and the Heun predictor; lb_correct:
 * LB predictor-corrector and the Heun corrector), 5 with Gauss-Seidel
 * coupling (field, force, lb, predict, correct), 3 with flow off (field,
 * predict, correct).  Errors: LCBP_EINVAL if capacity < *nkernels.
 */
LCBP_API int lcbp_profile_steps(lcbp_lattice *h, int nsteps, double *kernel_ms, int capacity, int *nkernels);

/*
 * Kernel selection.  LCBP_PATH_AUTO (default) runs the fast path -- two
 * z-marching kernels that stage planes in shared memory with TMA tile loads
 * -- whenever flow is on, coupling is Jacobi and nx is a multiple of 4;
 * otherwise, or with LCBP_PATH_GENERIC, three one-thread-per-site kernels.
 * FP32 fast kernels come in two builds, one or two lattice sites per thread
 * (the latter on packed FP32x2 arithmetic); AUTO times both, LCBP_PATH_FAST1
 * and LCBP_PATH_FAST2 pin one (a lattice with walls runs one site per thread
 * under either).  All compute the same step.  Errors:
 * LCBP_EINVAL (unknown path, or LCBP_PATH_FAST2 on an FP64 lattice).
 */
LCBP_API int lcbp_set_path(lcbp_lattice *h, int path);

/*
 * *fast = 1 if the next step runs the fast path; *planes_per_cta = the
 * autotuned number of z-planes each CTA marches through and
 * *sites_per_thread = the autotuned 1 or 2 (both 0 before the first step, or
 * on the generic path).  The tuning times each candidate once per lattice
 * shape and dtype, writing scratch buffers only; AUTO results persist in the
 * file named by the environment variable LCBP_AUTOTUNE_CACHE, if set
 * (lines "nx ny nz dtype planes sites planes_q", dtype + 100 for a lattice
 * with walls; see lcbp_get_tuning for the last two fields; a line without
 * planes_q gives both kernels the same planes).  Any pointer may be NULL.
 */
LCBP_API int lcbp_get_path(lcbp_lattice *h, int *fast, int *planes_per_cta, int *sites_per_thread);

/*
 * The fast path's tuning in full: each of the two kernels has its own planes
 * per CTA and sites per thread.  *planes_per_cta and *spt_lb = those of the
 * LB / Heun-corrector kernel (what lcbp_get_path reports), *planes_per_cta_q
 * and *spt_q = those of the molecular-field / stress / predictor kernel; all
 * 0 before the first step or on the generic path.  The autotune cache line
 * holds spt_lb + 10 * spt_q in its sites field and planes_per_cta_q after it.
 * Any pointer may be NULL.
 */
LCBP_API int lcbp_get_tuning(lcbp_lattice *h, int *planes_per_cta, int *spt_lb, int *spt_q, int *planes_per_cta_q);

/*
 * Copy out the Beris-Edwards rate dQ/dt = R(Q, u) = Gamma H + S(W, Q) - u.grad Q
 * of the current state (Sec. 2.1 Eq. Qevolution, mat_der; central differences,
 * trace of S removed, u from f, or u = 0 with flow off): 5 * N values.
 * Errors: LCBP_EINVAL, LCBP_ESTATE (flow on and f never initialised).
 */
LCBP_API int lcbp_read_rate(lcbp_lattice *h, void *dst, int dtype);

/*
 * Reset f to the equilibrium f^eq(rho, u, sigma_LC(Q)) of the current moments
 * and the current Q (used when plain stepping resumes after Q was advanced
 * by other means, e.g. the learned surrogate).  Errors: LCBP_ESTATE.
 */
LCBP_API int lcbp_reequilibrate_f(lcbp_lattice *h);

/* Synchronise the lattice's stream.  Errors: LCBP_ECUDA; LCBP_ETIMEOUT if a
 * bounded device-side wait of the fast path gave up (results invalid). */
LCBP_API int lcbp_synchronize(lcbp_lattice *h);

/*
 * Self-test of the bounded device-side wait that every barrier wait of the
 * fast kernels uses.  One CTA on the current device waits, for at most
 * limit_ms milliseconds (0 < limit_ms <= 1000), on a shared-memory barrier
 * that nothing arrives on.  *timed_out is set to 1 when the wait gave up
 * and reported it to the host, as the fast kernels' waits do before the
 * stepping calls return LCBP_ETIMEOUT; the CUDA context stays usable.
 * Not part of the method; no lattice is needed.  Errors: LCBP_EINVAL (bad
 * limit or NULL), LCBP_ECUDA.
 */
LCBP_API int lcbp_check_wait_timeout(double limit_ms, int *timed_out);

/* Copy out Q (5 * N), u (3 * N), rho (N) or f (15 * N) values.  Errors: LCBP_EINVAL. */
LCBP_API int lcbp_read_q(lcbp_lattice *h, void *dst, int dtype);
LCBP_API int lcbp_read_u(lcbp_lattice *h, void *dst, int dtype);
LCBP_API int lcbp_read_rho(lcbp_lattice *h, void *dst, int dtype);
LCBP_API int lcbp_read_f(lcbp_lattice *h, void *dst, int dtype);

/*
 * Total lattice free energy F_h = sum_x f_h(x), the per-site density in the
 * state's precision and the sum over sites in FP64 on the device, with the
 * lattice density
 *   f_h = bulk(Q) + (K/2) sum_g |D+_g Q|^2 + 2 K q0 Q:(eps D0 Q) + 2 K q0^2 |Q|^2
 * whose exact gradient is -H (Sec. 2.1 Eq. free_energy).
 * Errors: LCBP_ENONFINITE if Q holds NaN/Inf.
 */
LCBP_API int lcbp_free_energy(lcbp_lattice *h, double *F);

/* Sum of rho and of rho u over the lattice (sums over sites in FP64 on the device).  LCBP_ENONFINITE on NaN/Inf. */
LCBP_API int lcbp_totals(lcbp_lattice *h, double *mass, double momentum[3]);

/*
 * Fraction of sites whose scalar order q (largest eigenvalue of Q, Sec. 2.1)
 * is below `threshold` (the paper uses 0.19 to mark disclinations).  Each
 * site is decided as in FP64 (Sylvester's criterion on threshold I - Q).
 */
LCBP_API int lcbp_defect_fraction(lcbp_lattice *h, double threshold, double *fraction);

/*
 * Polarised-light texture (Sec. 2.3, rendering of the optical pattern): the
 * transmitted intensity S_0 of unpolarised light of unit intensity that
 * passes a linear polariser at phi_in, the lattice planes z = 0 .. Nz-1 in
 * turn (each a uniaxial retarder of thickness h: director = unit eigenvector
 * of the largest eigenvalue q of Q, beta = atan2(d_x, d_y), retardance
 * delta = 2 pi q h / lambda (n_o n_e / sqrt(n_o^2 sin^2 alpha +
 * n_e^2 cos^2 alpha) - n_o), cos alpha = d_z), and an analyser at phi_out;
 * the image is the weighted sum over the wavelengths.  Polariser angles enter
 * the Mueller matrices as 2 phi, so phi_in = 0, phi_out = pi/2 is the crossed
 * pair.  lcbp_optics_default fills the section's values: lambda = 16, 18,
 * 20 lattice units with weights 0.2, 0.6, 0.2, n_o = 1.5, n_e = 2.0, h = 1,
 * phi_in = 0, phi_out = pi/2.
 * img: caller-owned host buffer of Nx * Ny floats, [y][x].  Computed on the
 * GPU in FP32 from the current Q.  Errors: LCBP_EINVAL (NULL, nlambda outside
 * 1..4, a wavelength <= 0).
 */
typedef struct lcbp_optics {
  int nlambda;
  double lambda[4];
  double weight[4];
  double n_o, n_e, h;
  double phi_in, phi_out;
} lcbp_optics;
LCBP_API int lcbp_optics_default(lcbp_optics *o);
LCBP_API int lcbp_texture(lcbp_lattice *h, const lcbp_optics *o, float *img);

/*
 * Checkpoint: a versioned binary file with a header (magic, version, dims,
 * state dtype, parameters, step count) followed by the raw state in the state
 * type (deviation populations, moments, Q), so a resumed run is bitwise
 * identical to an uninterrupted one.
 * lcbp_load requires a lattice of the same dims and dtype.  Errors: LCBP_EIO,
 * LCBP_EINVAL (mismatch).
 */
LCBP_API int lcbp_save(lcbp_lattice *h, const char *path);
LCBP_API int lcbp_load(lcbp_lattice *h, const char *path);

/*
 * Raw snapshot of the state: the deviation populations f (15 N), the moments
 * [rho - 1, u] (4 N) and Q (5 N), all in the state type, with no conversion,
 * so that lcbp_restore brings back exactly (bitwise) the state of the moment
 * of the snapshot; the step counter is not part of it.  dst / src: host or
 * device memory of lcbp_snapshot_bytes(h) bytes, owned by the caller.  Both
 * calls synchronise the lattice's stream.  Errors: LCBP_EINVAL (NULL
 * pointers), LCBP_ESTATE (snapshot before f is initialised), LCBP_ECUDA.
 * The paper has no such call; it serves roll-back (the surrogate judge).
 */
LCBP_API size_t lcbp_snapshot_bytes(lcbp_lattice *h);
LCBP_API int lcbp_snapshot(lcbp_lattice *h, void *dst);
LCBP_API int lcbp_restore(lcbp_lattice *h, const void *src);

/* ------------------------------------------------------------------------
 * Batched replicas (parameter sweeps): R independent periodic lattices of
 * uneven sizes, each with its own Landau-de Gennes and kinetic parameters,
 * advanced together.  Their fields are concatenated structure-of-arrays
 * blocks on one device, replicas of equal dims (a class) back to back.
 * Every kernel of a step is one launch over all replicas, and nsteps are
 * replayed from a captured CUDA graph.  Two kernel sets:
 *   fast (open when flow is on, coupling is Jacobi, every class has
 *     nx % 4 == 0 and there are at most 4 classes): the two z-marching TMA
 *     kernels of the single-lattice fast path, each field of a class read as
 *     one 5-D tensor; each kernel's planes per CTA are picked per class by
 *     timing candidates; FP32 classes whose last 32-column tile would be at
 *     most half full (nx % 32 in 1..16) run tiles of 16 x 16 sites;
 *   generic: persistent CTAs walking one tile work-list that spans all
 *     replicas; the tile shape is picked by timing candidate shapes.
 * LCBP_PATH_AUTO (default) tunes both where the fast set is open and runs
 * the faster; LCBP_PATH_FAST1 runs the fast set wherever it is open;
 * LCBP_PATH_GENERIC always the generic set.  Tuning happens at the first
 * lcbp_batch_step after creation or a path change and writes scratch
 * buffers only.  Each replica computes exactly what a lattice of its own
 * computes with the same kernel set (one site per thread on the fast set).
 * ------------------------------------------------------------------------ */
typedef struct lcbp_batch lcbp_batch;

/* Per-replica parameters (meanings as in lcbp_set_ldg / lcbp_set_flow). */
typedef struct lcbp_params {
  double A0, gamma, K, q0; /* Sec. 2.1 Eq. (free_energy) */
  double tau_f, xi, Gamma; /* Sec. 2.1, 2.2 kinetics */
} lcbp_params;

/*
 * Fills *out from the reduced chirality kappa and temperature tau of Sec. 2.1
 * (gamma = 27 / (9 + tau), K = kappa^2 A0 gamma / (108 q0^2), as
 * lcbp_set_ldg_kappa_tau) and the kinetic parameters.  Errors: LCBP_EINVAL
 * (NULL out, tau <= -9, q0 == 0, kappa < 0, non-finite values).
 */
LCBP_API int lcbp_params_kappa_tau(double A0, double q0, double kappa, double tau, double tau_f, double xi,
                                   double Gamma, lcbp_params *out);

/*
 * dims: 3 * R ints (nx, ny, nz of replica r, each >= 1); params: R entries.
 * Flow on, Jacobi coupling; Q = 0, f unset.  Errors: LCBP_EINVAL, LCBP_ENOMEM.
 */
LCBP_API int lcbp_batch_create(int R, const int *dims, const lcbp_params *params, int state_dtype, lcbp_batch **out);
LCBP_API int lcbp_batch_destroy(lcbp_batch *b);
/* flow_on / coupling for all replicas (as lcbp_set_flow). */
LCBP_API int lcbp_batch_set_flow(lcbp_batch *b, int flow_on, int coupling);
/* Initial Q of replica r (as lcbp_init_q; the slab helix uses replica r's gamma). */
LCBP_API int lcbp_batch_init_q(lcbp_batch *b, int r, int kind, double amplitude, double noise, uint64_t seed,
                               const int *region);
/* Upload Q of replica r (5 * n_r values, boundary layout). */
LCBP_API int lcbp_batch_set_q(lcbp_batch *b, int r, const void *q5, int dtype);
/* f = f^eq(rho0, u = 0, sigma_LC(Q)) in every replica. */
LCBP_API int lcbp_batch_init_f_equilibrium(lcbp_batch *b, double rho0);
/* Advance every replica by nsteps (enqueued; graph replay). */
LCBP_API int lcbp_batch_step(lcbp_batch *b, int nsteps);
LCBP_API int lcbp_batch_synchronize(lcbp_batch *b);
/* Per-replica reads and FP64 diagnostics (as the lattice versions). */
LCBP_API int lcbp_batch_read_q(lcbp_batch *b, int r, void *dst, int dtype);
LCBP_API int lcbp_batch_read_u(lcbp_batch *b, int r, void *dst, int dtype);
LCBP_API int lcbp_batch_free_energy(lcbp_batch *b, int r, double *F);
LCBP_API int lcbp_batch_totals(lcbp_batch *b, int r, double *mass, double momentum[3]);
LCBP_API int lcbp_batch_defect_fraction(lcbp_batch *b, int r, double threshold, double *fraction);
/*
 * Kernel selection for the batch: LCBP_PATH_AUTO (default), LCBP_PATH_FAST1
 * or LCBP_PATH_GENERIC (see above).  Waits for the batch's stream, drops its
 * graph; the next lcbp_batch_step retunes.  Errors: LCBP_EINVAL (other paths).
 */
LCBP_API int lcbp_batch_set_path(lcbp_batch *b, int path);
/* *fast = 1 if steps run the fast kernels; *planes_per_cta = the LB /
 * Heun-corrector kernel's tuned z-chunk (tuned per class and per kernel; the
 * first class's value), 0 before the first step or on the generic path.
 * Either may be NULL. */
LCBP_API int lcbp_batch_get_path(lcbp_batch *b, int *fast, int *planes_per_cta);
/* R, total sites, tuned tile shape (tx, ty, tz) and persistent CTAs per launch
 * of the generic path, steps done. */
LCBP_API int lcbp_batch_get_info(lcbp_batch *b, int *R, long long *total_sites, int tile[3], int *persistent_ctas,
                                 long long *step);

/* ------------------------------------------------------------------------
 * Allocation-free free energy.  For callers that cannot allocate device
 * memory when they need the free energy -- code whose framework allocator
 * owns the device heap, real-time loops that must not touch an allocator --
 * this computes F_h of a caller-owned device Q field without any cudaMalloc,
 * cudaFree or other allocating call.  It covers a periodic lattice with the
 * one-constant energy: it equals lcbp_free_energy of a lattice without walls
 * and with L2 = K (no lcbp_set_walls, no lcbp_set_l2).  Its scratch, the
 * per-block partial sums of the FP64 reduction (32.8 KB), is a fixed device
 * array that every GPU loading the library holds until exit.
 *   q5: device pointer, 5 * N values in the layout above (dtype LCBP_F32 or
 *       LCBP_F64); A0, gamma, K, q0: as lcbp_set_ldg; stream: a cudaStream_t
 *       (NULL = legacy default stream).  *F receives the result: the call
 *       copies it to host memory and synchronises the stream.
 * The first call in each CUDA context of a device looks up the array's device
 * address there (again after cudaDeviceReset); make that first call before
 * any stream capture begins.  All calls share the one array (its contents are
 * those of the last call; every slot is rewritten by each call, so nothing
 * needs clearing), hence calls that overlap on the GPU -- from several
 * threads or streams at once -- race.
 * Errors: LCBP_EINVAL (NULL pointers, bad dtype, sizes < 1, more than
 * LCBP_NOALLOC_MAX_SITES sites), LCBP_ENONFINITE, LCBP_ECUDA.
 * There is no counterpart of this call in the paper.
 * ------------------------------------------------------------------------ */
#define LCBP_NOALLOC_MAX_SITES (1LL << 31)
LCBP_API int lcbp_free_energy_noalloc(const void *q5, int dtype, int nx, int ny, int nz, double A0, double gamma,
                                      double K, double q0, void *stream, double *F);

/* ------------------------------------------------------------------------
 * Learned surrogate (not part of the paper's method): a periodic 3x3x3
 * convolutional network that advances Q by k solver steps (k = 10 unless
 * set) as a learned correction to k explicit Euler steps of the
 * Beris-Edwards rate R:
 *   x = [Q (5), u / s_u (3), kappa - 1, tau, R / s_r (5)]  ->  h0 = relu(conv x),
 *   4 x { a = relu(conv h);  h = h + conv a },  y = conv h (5 channels),
 *   Q(t + k) = Q(t) + k R(t) + s_dq * y,
 * with 32 hidden channels, BF16 weights and activations and FP32
 * accumulation on tcgen05 tensor cores (forward, backward-data and weight
 * gradients), masked MSE loss and Adam.  A surrogate object is built
 * for one lattice size.  Parameters cross the boundary as one FP32 vector:
 * for each layer in the order in, b0a, b0b, ..., b3a, b3b, out the weights
 * W[t][c_in][c_out] (t = 9 (dz+1) + 3 (dy+1) + (dx+1), tap offset (dx, dy, dz),
 * y(r) = b + sum_t W_t^T x(r + o_t)) followed by the bias b[c_out].
 * ------------------------------------------------------------------------ */
typedef struct lcbp_surrogate lcbp_surrogate;

/* Number of FP32 values of the parameter vector (238757). */
LCBP_API size_t lcbp_surrogate_param_count(void);
/* Surrogate for an nx * ny * nz lattice; training != 0 also allocates the
 * activations, gradients and Adam state.  Parameters start at zero. */
LCBP_API int lcbp_surrogate_create(int nx, int ny, int nz, int training, lcbp_surrogate **out);
LCBP_API int lcbp_surrogate_destroy(lcbp_surrogate *s);
/* Input scales s_u (velocity, default 1e-3) and s_r (rate, default 1e-3) and
 * the output scale s_dq (default 1e-3). */
LCBP_API int lcbp_surrogate_set_scales(lcbp_surrogate *s, double s_u, double s_r, double s_dq);
/* Convolution kernel: LCBP_CONV_AUTO (default) stages each input plane once
 * per 128-site tile and serves all 27 taps from it (the "window" kernel)
 * where that window fits shared memory (nx <= 101), else loads one shifted
 * tile per tap (LCBP_CONV_TAPS).  LCBP_CONV_WINDOW
 * requires the window kernel (LCBP_EINVAL where it does not fit).  Both
 * compute the same sums (FP32 accumulation in a different order).
 * OR-ing LCBP_CONV_DW_CUDA_CORES into the kind moves the weight gradients of
 * training from the tensor-core kernel (used where its staged plane windows
 * fit shared memory, nx <= 177) to the CUDA-core kernel (FP32 atomics, not
 * bitwise reproducible); both compute the same sums. */
#define LCBP_CONV_AUTO 0
#define LCBP_CONV_TAPS 1
#define LCBP_CONV_WINDOW 2
#define LCBP_CONV_DW_CUDA_CORES 4
LCBP_API int lcbp_surrogate_set_conv_kernel(lcbp_surrogate *s, int kind);
/* Upload / download the parameter vector (host or device FP32; Adam state is reset on upload). */
LCBP_API int lcbp_surrogate_set_params(lcbp_surrogate *s, const float *params, size_t count);
LCBP_API int lcbp_surrogate_get_params(lcbp_surrogate *s, float *params, size_t count);
/*
 * Weights file of a trained network: save writes the parameter vector and the
 * input / output scales to `path`, load reads them back into a surrogate
 * (any lattice size: the weights do not depend on it; Adam state is reset).
 * Format, version 1, little-endian: "LCBPSURR", int32 version, int32 residual
 * blocks (4), width (32), input channels (15), output channels (5), kernel
 * size (3), solver steps per call k, int32 0, double s_u, s_r, s_dq,
 * uint64 count, then count FP32 parameters in the order above.
 * Errors: LCBP_EINVAL (NULL path; a file of another architecture), LCBP_EIO
 * (cannot open, not a version-1 file, truncated), LCBP_ENONFINITE
 * (non-finite parameters).  Not in the paper (the surrogate is an addition).
 */
LCBP_API int lcbp_surrogate_save(lcbp_surrogate *s, const char *path);
LCBP_API int lcbp_surrogate_load(lcbp_surrogate *s, const char *path);
/* Gradient of the last training step's loss, in the parameter-vector layout. */
LCBP_API int lcbp_surrogate_get_grads(lcbp_surrogate *s, float *grads, size_t count);
/* Network output y (5 * N values, [c][z][y][x]) for fields Q (5 * N), u (3 * N,
 * NULL = 0) and rate R (5 * N, NULL = 0) in the same dtype. */
LCBP_API int lcbp_surrogate_forward(lcbp_surrogate *s, const void *q5, const void *u3, const void *r5, double kappa,
                                    double tau, int dtype, float *y5);
/* Solver steps k that one call stands for (1..1000; default 10).  Set it
 * before training: the network learns the correction to k Euler steps. */
LCBP_API int lcbp_surrogate_set_steps(lcbp_surrogate *s, int k);
LCBP_API int lcbp_surrogate_get_steps(lcbp_surrogate *s, int *k);
/* ncalls times: R = R(Q, u) of the lattice (FP32 state, same size), then
 * Q += k R + s_dq * net(Q, u, kappa, tau, R).  u is not advanced and f is left
 * as it was: call lcbp_reequilibrate_f before plain stepping resumes. */
LCBP_API int lcbp_surrogate_step(lcbp_surrogate *s, lcbp_lattice *h, double kappa, double tau, int ncalls);
/* One Adam step (learning rate lr) on the masked MSE between y and
 * (dq5 - k R) / s_dq (dq5: the true k-step change of Q, 5 * N values; mask:
 * N values or NULL); *loss receives the loss. */
LCBP_API int lcbp_surrogate_train_step(lcbp_surrogate *s, const void *q5, const void *u3, const void *r5,
                                       double kappa, double tau, const void *dq5, const void *mask, int dtype,
                                       double lr, double *loss);

/* ------------------------------------------------------------------------
 * Judged surrogate run (not in the paper: the judge and fallback of the
 * learned surrogate, with the plain solver of Sec. 2.2 as the judge).
 *
 * The judge advances a lattice (FP32, periodic, the surrogate's size) in
 * segments of calls_per_segment surrogate calls of k solver steps each (k of
 * the surrogate, lcbp_surrogate_set_steps, fixed when the judge is made).  A
 * segment starts from a raw snapshot of the state (lcbp_snapshot).  After
 * its calls f is re-equilibrated to the new Q (lcbp_reequilibrate_f); then one
 * more surrogate call, on a copy of that state, is compared with k plain
 * steps of the lattice: the segment stands if
 *   |F_sur - F_plain| / |F_plain| <= tol_F   and, if tol_Q > 0,
 *   max |Q_sur - Q_plain| <= tol_Q,
 * and the k plain steps count as time advanced.  Otherwise (or if the state
 * became non-finite) the snapshot is restored and the segment is redone with
 * plain steps, so a run that never accepts a segment equals a plain run
 * bitwise.  The first warmup_steps of the run, and the end where fewer than
 * 2k steps remain, are stepped plainly.
 * Time t starts at 0 when the judge is created.
 * ------------------------------------------------------------------------ */
typedef struct lcbp_judge lcbp_judge;
typedef struct lcbp_judge_config {
  double kappa, tau;      /* the surrogate's conditioning (Sec. 2.1 reduced chirality, temperature) */
  int calls_per_segment;  /* M >= 1 */
  double tol_F;           /* >= 0 */
  double tol_Q;           /* <= 0: Q is not judged */
  long long warmup_steps; /* plain steps before the first segment (the fast initial relaxation) */
} lcbp_judge_config;
typedef struct lcbp_judge_stats {
  long long t;                /* steps advanced */
  long long segments, accepted, fallbacks;
  long long surrogate_calls;  /* calls kept (ten steps each) */
  long long plain_steps;      /* plain steps kept (judge steps and redone segments) */
  double last_gap_F, last_gap_Q;  /* of the last judgement (NaN if it failed) */
  double max_gap_F;           /* largest accepted relative F gap */
  double mean_gap_F, mean_gap_Q;  /* over the judgements with finite gaps */
  long long judged;           /* judgements with finite gaps */
} lcbp_judge_stats;

/* The judge keeps both handles (the caller keeps them alive and owns them)
 * and allocates two snapshots and a scratch lattice of the lattice's size.
 * Errors: LCBP_EINVAL (NULL pointers, calls_per_segment < 1, tol_F < 0,
 * non-finite values), LCBP_ENOMEM. */
LCBP_API int lcbp_judge_create(lcbp_lattice *h, lcbp_surrogate *s, const lcbp_judge_config *c, lcbp_judge **out);
LCBP_API int lcbp_judge_destroy(lcbp_judge *j);
/*
 * Advance to time t_end.  With log_every > 0 (a multiple of k; t_end then a
 * multiple of k too) the free energy F_h (lcbp_free_energy) and the defect
 * fraction for defect_threshold (lcbp_defect_fraction) are logged at every
 * multiple of log_every passed, from the state the run keeps, into log_t,
 * log_F, log_defect (capacity entries each); *nlog receives the count.
 * Errors: LCBP_EINVAL (bad log_every or t_end, arrays too small), and those of
 * the calls it makes other than LCBP_ENONFINITE, which fails a judgement.
 */
LCBP_API int lcbp_judge_advance(lcbp_judge *j, long long t_end, int log_every, double defect_threshold,
                                long long *log_t, double *log_F, double *log_defect, int capacity, int *nlog);
LCBP_API int lcbp_judge_get_stats(lcbp_judge *j, lcbp_judge_stats *out);

#ifdef __cplusplus
}
#endif

#endif /* LCBP_H */
