/*
 * fsib.h - C ABI of the GB300 (sm_103a) Fourier spectral immersed boundary step.
 *
 * Method: Chen & Peskin, "A Fourier spectral immersed boundary method with exact
 * translation invariance, improved boundary resolution, and a divergence-free
 * velocity field" (arXiv 2302.08694). Section and equation names below refer to
 * that paper.
 *
 * ---------------------------------------------------------------------------
 * Conventions shared by every entry point
 * ---------------------------------------------------------------------------
 * Box.      Periodic box [0, L)^d with L = 1, d in {2, 3}.
 * Modes.    N Fourier modes per axis, N even, N >= 4. Integer modes per axis are
 *           m = -N/2 .. N/2-1 (Eq. kNh) and k = 2*pi*m/L. The unpaired mode
 *           m = -N/2 is held at zero in every spectral array (inputs: ignored;
 *           outputs: written as 0), so the kept set is symmetric and every field
 *           is real.
 * Spectral arrays ("half spectrum", as the spectrum of a real field):
 *           component-major, then (m_z,) m_y in FFT order (index i holds
 *           m = i for i < N/2, m = i - N otherwise), then m_x = 0 .. N/2-1.
 *           d = 3: [d][N][N][N/2] complex; d = 2: [d][N][N/2] complex.
 *           Complex numbers are interleaved (re, im). Element type: double in
 *           FSIB_FP64 mode, float in FSIB_MIXED mode.
 *           Represented field: u-hat(m) = H(m) for m_x > 0, conj(H(-m)) for
 *           m_x < 0, and the Hermitian part (H(m) + conj(H(-m)))/2 on m_x = 0.
 * Points.   X, F, U, omega are double, structure of arrays: [d][M] (row a is
 *           coordinate a, a = 0 is x). X is kept unwrapped; transforms use
 *           X mod L, force laws use plain differences.
 * Pointers. Every array argument may be device memory or host memory (pageable
 *           or pinned). Host arrays are copied through staging buffers owned by
 *           the handle and the call returns after the results are back on the
 *           host. With device arrays the call is asynchronous on the handle's
 *           stream unless stated otherwise. The caller owns all array arguments.
 * Errors.   0 on success, a negative FSIB_E* code otherwise; fsib_last_error()
 *           gives the message. No entry point falls back to the CPU.
 */
#ifndef FSIB_H
#define FSIB_H

#ifdef __cplusplus
extern "C" {
#endif

#define FSIB_OK            0
#define FSIB_EINVAL       -1  /* bad size, parameter, key or pointer */
#define FSIB_ENOMEM       -2  /* device allocation failed */
#define FSIB_ECUDA        -3  /* a CUDA call or kernel launch failed */
#define FSIB_ENONFINITE   -4  /* non-finite positions or velocities detected */
#define FSIB_ETIMEOUT     -5  /* a bounded device wait ran out */
#define FSIB_EUNSUPPORTED -6  /* valid request the library does not support */
#define FSIB_ESTATE       -7  /* call out of order (e.g. no force model set) */

#define FSIB_FP64  0          /* transforms and fluid solve in double */
#define FSIB_MIXED 1          /* spread, FFT, fluid solve, interp in float;
                                 forces, positions, invariants in double */

typedef struct fsib_plan* fsib_t;

/* Create a handle for one problem.
 * N: modes per axis (even, 4..1024). d: 2 or 3. M: number of boundary points (>= 1).
 * The fine grid (sigma N points per axis, rounded up to a multiple of 8 with no prime
 * factor above 3) and the dealiasing grid (3N/2, rounded up to an even length with no
 * prime factor above 3) must each fit
 * the longest transform, 2048 points in 2D and 512 in 3D: at sigma = 2 that is
 * N <= 1024 in 2D and N <= 256 in 3D. A larger grid returns FSIB_EUNSUPPORTED.
 * mu: dynamic viscosity (> 0). rho: density; rho > 0 selects Navier-Stokes
 * (Algorithm 1, Eqs. spatial_1-4), rho <= 0 the quasi-static Stokes stepper
 * (Eq. stokeslet, same midpoint rule in time). dt: time step (> 0).
 * tol: requested relative accuracy of each NUFFT (1e-14 .. 1e-2); it fixes the
 * spreading-kernel width and shape (appendix A.3). Precision starts as
 * FSIB_FP64. Allocates every device workspace on the current device. */
int fsib_create(fsib_t* out, int N, int d, int M, double mu, double rho,
                double dt, double tol);

/* Release the handle and all its device memory. NULL is accepted. */
int fsib_destroy(fsib_t h);

/* Stream (a cudaStream_t) on which later calls enqueue their work; NULL means
 * the legacy default stream. */
int fsib_set_stream(fsib_t h, void* stream);

/* Set a tuning or mode option; re-plans and re-allocates as needed. Keys:
 *  "precision"  0 = FSIB_FP64, 1 = FSIB_MIXED
 *  "sigma"      upsampling factor of the fine grid (1.5 .. 3, default 2)
 *  "width"      spreading-kernel width in fine cells (2 .. 16; 0 = from tol)
 *  "bin"        bin side in fine cells for the point sort (4 .. 32; 0 = auto)
 *  "native_fp64" FSIB_FP64 mode only: 0 = transforms in double-float arithmetic
 *               (pairs of floats, about 48 bits; default, fast on GB300's FP32
 *               pipes), 1 = transforms in FP64 arithmetic
 *  "graph"      1 = fsib_step replays a captured CUDA graph (default), 0 = direct launches
 *  "fft_tile", "fft_rows", "spread_slice": launch shapes, see fsib_autotune
 *  "check_finite" 1 = fsib_step checks positions for NaN/Inf at the end
 *               (adds a synchronisation), 0 = no check (default)
 *  "spread_sum" FSIB_MIXED gather spreads (appendix A.1, Eq. type1_conv): how each
 *               fine-grid cell sums its terms in FP32. 0 = plain FMAs; 1 = every
 *               term into a compensated (TwoSum) sum; 2 = the terms of each staged
 *               chunk of candidate points with FMAs, the chunk sums into a
 *               compensated sum (default). FSIB_FP64 mode ignores it.
 * Returns FSIB_EINVAL for an unknown key or out-of-range value. */
int fsib_set_option(fsib_t h, const char* key, double value);

/* Query a planned value. Keys: "nf" (fine grid per axis), "width", "beta",
 * "Nt" (dealiasing grid per axis), "precision", "bin", "workspace_bytes",
 * "launches_per_step" (kernels one fsib_step step enqueues). */
int fsib_get_info(fsib_t h, const char* key, double* value);

/* Closed-curve Hookean tension, d = 2 (Eq. elstic_force_2d):
 * F_i = K (X_{i+1} + X_{i-1} - 2 X_i)/dtheta^2, dtheta = 2*pi/M, weight omega = dtheta.
 * Points are ordered along the curve; the curve is closed. */
int fsib_set_force_curve(fsib_t h, double K);

/* Triangulated membrane with cot-weight springs, d = 3 (Sec. 6.2.3):
 * K_AB = (sigma/2)(cot C1 + cot C2) from the reference configuration Xref
 * ([3][M] double), F_i = sum_j K_ij (X_j - X_i), omega = 1 (nodal forces).
 * tri: [ntri][3] int32 vertex indices, counter-clockwise seen from outside
 * (used for the enclosed volume). Both arrays are copied; host or device. */
int fsib_set_force_mesh(fsib_t h, const int* tri, int ntri, const double* Xref,
                        double sigma);

/* Surface tension, d = 3 (Sec. 6.2.4): energy gamma S with S the summed triangle
 * areas, so F_i = -(gamma/2) sum over the triangles (i, j, k) at node i of
 * (X_j - X_k) x n_ijk, n_ijk the unit normal of (X_i, X_j, X_k); omega = 1 (nodal
 * forces). tri: [ntri][3] int32, counter-clockwise seen from outside (also used
 * for the enclosed volume); host or device, copied. fsib_invariants reports
 * E_p = gamma S. FSIB_EINVAL for d != 3, bad or repeated indices in a triangle,
 * or a non-finite gamma; fsib_step_adjoint rejects this model (FSIB_EUNSUPPORTED). */
int fsib_set_force_tension(fsib_t h, const int* tri, int ntri, double gamma);

/* Target-point springs, any d (Sec. 5.2.2, the Poiseuille channel walls):
 * F_i = K (X~_i - X_i) with weight omega (the Lagrangian meshwidth), so
 * c_i = omega K (X~_i - X_i). Xtarget: [d][M] double, host or device, copied.
 * Points need not form a closed curve; fsib_invariants then reports area or
 * volume 0 (unless a mesh was set in 3D) and E_p = (omega K/2) sum |X~ - X|^2.
 * Returns FSIB_EINVAL for a non-finite K or omega <= 0. fsib_step_adjoint
 * rejects this model (FSIB_EUNSUPPORTED). */
int fsib_set_force_target(fsib_t h, const double* Xtarget, double K, double omega);

/* Uniform body force density f0 (host array of d doubles; Sec. 5.2.2), added
 * to the Fourier coefficient f-hat(0) in every Navier-Stokes substep
 * (fsib_step and fsib_fluid_step). Zero by default. FSIB_EUNSUPPORTED for a
 * quasi-static Stokes handle (rho <= 0), FSIB_EINVAL for non-finite entries. */
int fsib_set_body_force(fsib_t h, const double* f);

/* Weighted force c_j = omega_j F_j of the current force model at X ([d][M]),
 * written to c ([d][M] double). */
int fsib_force(fsib_t h, const double* X, double* c);

/* Type-1 NUFFT spread (Eq. force_spreading_quad; appendix A.1):
 * f-hat(k) = L^-d sum_j omega_j F_j exp(-i k . X_j), k in K_N.
 * X, F: [d][M] double. omega: [M] double, or NULL for omega_j = 1.
 * fhat: half-spectrum output. Accuracy: the plan's tol, relative in the 2-norm. */
int fsib_spread(fsib_t h, const double* X, const double* F, const double* omega,
                void* fhat);

/* Type-2 NUFFT interpolation (Eq. velo_intp_fini; appendix A.2):
 * U_j = sum_{k in K_N} u-hat(k) exp(i k . X_j). uhat: half spectrum;
 * X, U: [d][M] double. */
int fsib_interp(fsib_t h, const void* uhat, const double* X, double* U);

/* Fluid update in Fourier space.
 * Navier-Stokes (rho > 0): with f-hat = fhat and u-hat^m = uhat on input,
 *   u-hat^{m+1/2} = (dt/2 V(f, u^m) + u^m)/(1 + mu dt |k|^2/(2 rho))        (Eq. spatial_2)
 *   u-hat^{m+1}   = (dt V(f, u^{m+1/2}) + (1 - mu dt|k|^2/(2 rho)) u^m)/(1 + mu dt |k|^2/(2 rho))  (Eq. spatial_3)
 *   with V(f, u) = P_k (f/rho - s-hat(u)) (Algorithm 2), s-hat the
 *   three-halves dealiased nonlinear term (Eq. nonlinear_kspace).
 *   uhat is overwritten with u-hat^{m+1}; uhat_half (may be NULL) receives u-hat^{m+1/2}.
 * Stokes (rho <= 0): uhat = mu^-1 (I/|k|^2 - k k^T/|k|^4) fhat, uhat(0) = 0
 *   (Eq. stokeslet); uhat_half is ignored. */
int fsib_fluid_step(fsib_t h, const void* fhat, void* uhat, void* uhat_half);

/* Advance nsteps time steps in place.
 * Navier-Stokes: state (X^m, u-hat^m, U^m) -> (X^{m+n}, u-hat^{m+n}, U^{m+n}) by
 *   Algorithm 1, where U^m must equal the interpolated velocity u^m(X^m)
 *   (fsib_interp gives U^0). U^{m+1} is interpolated at X^{m+1} after the
 *   position update, from a fine grid computed only near the windows at
 *   X^{m+1/2} (within one box of 8 fine cells): a point that moves farther in
 *   half a step (far beyond a stable dt) gets NaN in U^{m+1} and the handle
 *   records it. The first fsib_step, fsib_interp or fsib_invariants call that
 *   starts after the GPU has finished that step returns FSIB_ENONFINITE (and
 *   clears the record) without running; a synchronous step (host arrays, or
 *   "check_finite" set) returns it at once.
 * Stokes: X^{m+1} = X^m + dt U(X^{m+1/2}), X^{m+1/2} = X^m + dt/2 U(X^m),
 *   U(X) = interp(Stokeslet(spread(F(X), X)), X); uhat and U may be NULL
 *   (when given, U receives U(X^{m+1/2}) of the last step).
 * Host arrays are copied to device buffers before the steps and back after them.
 * For one Navier-Stokes step (nsteps = 1) on a page-locked host uhat, uhat is
 * copied inside the step instead, beside work that does not read it (the
 * force, the sort and the type-1 NUFFT; the final interpolations), so the
 * copies cost less than their transfer time. Synchronous when any array is
 * on the host.
 * Needs a force model. */
int fsib_step(fsib_t h, double* X, void* uhat, double* U, int nsteps);

/* Velocity gradient at the points: G[b][a][j] = d u_a/d x_b (X_j) for the field of
 * uhat (half spectrum), i.e. the type-2 sums of i k_b u-hat_a (Eq. velo_intp_fini
 * applied to the gradient). X: [d][M]; G: [d][d][M] double. */
int fsib_interp_grad(fsib_t h, const void* uhat, const double* X, double* G);

/* Reverse mode of K quasi-static Stokes steps (rho <= 0 handles only).
 * Given X0 ([d][M]) and dL/dX^K ([d][M]) for the state after K steps of fsib_step,
 * writes dL/dX^0 ([d][M]) and dL/dsigma (one double), sigma being the stiffness of
 * the force model (K of the curve, sigma of the mesh; the force is linear in it).
 * The velocity U(X) = interp(Stokeslet(spread(X, c(X))), X) has the transpose
 * Jacobian J^T lam = (grad u)^T lam + (grad w)^T c + c(w), where w is the velocity
 * of lam used as forces (spread and interp are adjoint, Sec. 4.4) and c(.) the
 * (linear, symmetric) force law; a step X1 = X + dt U(X + dt/2 U(X)) is reversed as
 * a = dt J(X_half)^T lam1, lam0 = lam1 + a + dt/2 J(X)^T a. Forward states are kept
 * every ckpt_every steps and recomputed segment by segment. Allocates its
 * checkpoint buffers on first use. */
int fsib_step_adjoint(fsib_t h, const double* X0, int K, int ckpt_every, const double* dLdXK,
                      double* dLdX0, double* dLdsigma);

/* Diagnostics in double, synchronous (Sec. 4). out[0] enclosed volume (d = 3,
 * needs the mesh) or area (d = 2, curve order), out[1] elastic energy E_p,
 * out[2] kinetic energy E_K = rho/2 L^d sum |u-hat|^2 (rho = 1 for Stokes),
 * out[3] |u-hat(0)|, out[4] max_k |k . u-hat(k)|/|k| over max_k |u-hat(k)|,
 * out[5] dissipation mu L^d sum |k|^2 |u-hat|^2. uhat may be NULL (out[2..5] = 0).
 * Returns FSIB_ENONFINITE if X or uhat holds NaN/Inf. */
int fsib_invariants(fsib_t h, const double* X, const void* uhat, double out[6]);

/* Pressure (Eq. pressure_poisson_k): p-hat = -i k.(f-hat - rho s-hat(u-hat))/|k|^2,
 * p-hat(0) = 0 (mean-free pressure), unpaired modes -N/2 zero. fhat, uhat: half
 * spectra of the plan ([d][...]); phat: one half-spectrum component
 * ([(N)][N][N/2]). s-hat is the dealiased nonlinear term of the Navier-Stokes
 * update; it is dropped for a Stokes handle or uhat == NULL (rho s-hat = 0).
 * The pressure at points follows from fsib_interp of a spectrum whose first
 * component is phat. */
int fsib_pressure(fsib_t h, const void* fhat, const void* uhat, void* phat);

/* Channel flux (Eq. poiseuille_flux), synchronous: the velocity component
 * `comp` averaged over the axes other than `axis`, integrated over the band
 * y0 <= x_axis <= y1: *flux = int_{y0}^{y1} ubar(y) dy, computed from the
 * modes m e_axis of uhat (half spectrum) with the exact integral of each
 * exponential. comp, axis in [0, d); flux is a host pointer. Returns
 * FSIB_EINVAL for bad indices or non-finite limits, FSIB_ENONFINITE for a
 * non-finite result. */
int fsib_band_flux(fsib_t h, const void* uhat, int comp, int axis, double y0, double y1,
                   double* flux);

/* Launch-shape options, exact reorderings that leave results unchanged to
 * rounding: "fft_tile" (4, 8, 16: lines per strided-pass tile), "fft_rows"
 * (2, 4, 8: row pairs per CTA in the row passes), "spread_slice" (128..4096:
 * candidate points per slice of a 3D gather box). fsib_autotune picks them by
 * timing whole steps on copies of the given state (X, uhat, U as for fsib_step;
 * the arguments are not modified), one option at a time over the values above.
 * Synchronous. Not an operation of the paper: a library service. */
int fsib_autotune(fsib_t h, const double* X, const void* uhat, const double* U);

/* Batches of independent problems (uneven N, d, M), advanced together.
 * fsib_batch_create makes one member handle per problem (arrays of length
 * nprob; precision FSIB_FP64 or FSIB_MIXED for all members). Set each member's
 * force model through fsib_batch_member. fsib_batch_step advances every member
 * by nsteps steps (as fsib_step) with one CUDA graph launch per step. The graph is
 * built from a recording of every member's step: members with the same sequence
 * of phases (same d, flow and arithmetic) form a group, and each phase runs as
 * one launch over the group's members (at most 16 a launch; the members'
 * arguments travel in the launch's parameter space). Members with the same d, N,
 * fine and dealiasing grids and step structure form a group; groups run as
 * concurrent branches of the graph. Double-float and FP64 transforms run once
 * per member. The graph is
 * rebuilt when the arrays or a member's plan, launch shapes or force model
 * change. X, uhat, U: arrays of nprob device pointers (uhat[i], U[i] may be
 * NULL for Stokes members). fsib_batch_autotune runs fsib_autotune on every
 * member. Info keys: "nprob", "launches_per_step" (kernel launches in one batch
 * step), "groups", "merge". */
typedef struct fsib_batch* fsib_batch_t;
int fsib_batch_create(fsib_batch_t* out, int nprob, const int* N, const int* d, const int* M,
                      const double* mu, const double* rho, const double* dt, const double* tol,
                      int precision);
int fsib_batch_member(fsib_batch_t b, int i, fsib_t* h);
/* Batch options. "merge": 1 (default) = each phase of the members' steps runs as one launch
 * over the members of a group that share its kernel (see fsib_batch_step); 0 = one graph
 * branch per member holding that member's own launches. "group_max": largest group (0 = no
 * limit, default; a larger group is split into balanced ones that run concurrently). Results
 * agree to rounding either way. FSIB_EINVAL for an unknown key or a bad value. */
int fsib_batch_set_option(fsib_batch_t b, const char* key, double value);
int fsib_batch_set_stream(fsib_batch_t b, void* stream);
int fsib_batch_autotune(fsib_batch_t b, double* const* X, void* const* uhat, double* const* U);
int fsib_batch_step(fsib_batch_t b, double* const* X, void* const* uhat, double* const* U,
                    int nsteps);
int fsib_batch_info(fsib_batch_t b, const char* key, double* value);
const char* fsib_batch_last_error(fsib_batch_t b);
int fsib_batch_destroy(fsib_batch_t b);

/* Per-launch-site profiling. When enabled, every call enqueues CUDA events
 * around each kernel launch site on the handle's stream and fsib_step launches
 * its kernels directly instead of replaying the captured graph. Entries
 * accumulate until fsib_profile_reset. For entry i (0 <= i < fsib_profile_count):
 * name (NUL-terminated, truncated to name_len), total milliseconds, number of
 * launches, and the algorithmic bytes and flops of one launch (each input read
 * once, each output written once; flops counted as 5 n log2 n per length-n
 * complex FFT line). fsib_profile_entry synchronises the handle's stream. */
int fsib_profile_enable(fsib_t h, int on);
int fsib_profile_reset(fsib_t h);
int fsib_profile_count(fsib_t h);
int fsib_profile_entry(fsib_t h, int i, char* name, int name_len, double* total_ms,
                       int* launches, double* bytes_per_launch, double* flops_per_launch);

/* Measured arithmetic peak of the current device for the roofline: kind 0 =
 * FP64 FMA throughput, kind 1 = FP32 FMA throughput, in GFLOP/s (an FMA counts
 * as 2 flops). Runs a short register-resident kernel; synchronous. */
int fsib_measure_peak(int kind, double* gflops);

/* Type-1 spread that allocates no device memory.
 * The paper has no counterpart: this is a library service. Some callers cannot
 * call cudaMalloc at all - code living inside a host framework whose caching
 * allocator owns all device memory, or latency-critical loops that cannot take
 * cudaMalloc's implicit device-wide synchronisation - and fsib_create allocates
 * its workspaces. This entry point computes the same transform as fsib_spread
 * (f-hat(k) = L^-d sum_j omega_j F_j exp(-i k . X_j), k in K_N, same layouts and
 * accuracy) with every scratch buffer (fine grid, FFT intermediates, point sort,
 * tables) carved from one file-scope device array of FSIB_STATIC_SCRATCH_BYTES
 * = 64 MiB, which every GPU that loads the library holds until the process exits.
 * It calls no cudaMalloc, cudaFree or allocating library routine.
 * X, F ([d][M] double), omega ([M] double or NULL) and fhat (half spectrum,
 * double or float complex per precision) must be device arrays; the work is
 * enqueued on `stream` (a cudaStream_t, NULL = legacy default stream).
 * Returns FSIB_EINVAL, with a message in fsib_static_last_error(), when the
 * problem needs more scratch than the array holds (e.g. 3D FP64 N > 48, or 3D
 * mixed N > 64 at moderate M) or an argument is invalid.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture. Every later call made outside stream capture looks the
 * address up again (after a device reset the array is new and empty).
 * The twiddle and deconvolution tables are built on the host and copied into the
 * array by the first call for a given (device, N, d, tol, precision), which waits
 * for that copy (a stream synchronisation); later calls with the same values
 * reuse them and enqueue kernels and memsets only. Under stream capture a call
 * whose tables are not there returns FSIB_EINVAL without enqueueing anything:
 * make one call with the same values outside capture first.
 * All calls share the one array, which keeps the previous call's contents (the
 * call clears what must start at zero; a call with other sizes replaces the
 * tables): calls that overlap on the GPU, from several streams or host threads,
 * race on it. */
int fsib_spread_static(int N, int d, int M, double tol, int precision, const double* X,
                       const double* F, const double* omega, void* fhat, void* stream);

/* Message of the last fsib_spread_static error on the calling host thread. */
const char* fsib_static_last_error(void);

/* Message of the last error on this handle ("" if none); h may be NULL for
 * errors of fsib_create. */
const char* fsib_last_error(fsib_t h);

/* Library version string. */
const char* fsib_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FSIB_H */
