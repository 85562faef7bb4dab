/*
 * cosmos.h -- C ABI of libcosmos_gb300.so: BSSN + perfect-fluid + massless-
 * scalar evolution on a periodic 3D grid, FP64, on one NVIDIA GB300 GPU.
 *
 * The calls follow the evolution problem of Yoo et al., "COSMOS: a numerical
 * relativity code specialized for PBH formation" (section "Physical system
 * settings"): the Einstein equations G = 8 pi T with T = T^SC + T^FL,
 * T^FL = (rho + P) u u + P g, P = w rho, box phi = 0 and div T^FL = 0,
 * integrated in the 3+1 (BSSN, chi-variant) form that the paper refers to
 * the standard textbooks for, from long-wavelength initial data whose fluid
 * density satisfies the Hamiltonian constraint (same section, last
 * paragraph); the fluid uses the Kurganov-Tadmor central scheme the paper
 * names.  Spatial derivatives are 4th-order centred finite differences with
 * 6th-derivative Kreiss-Oliger dissipation; time integration is classic RK4.
 *
 * Conventions (all calls):
 *  - Units G = c = 1.  Grid points x = x0 + (i, j, k) * h, periodic.
 *  - State layout: structure of arrays, double precision.  Field f of point
 *    (i, j, k) is state[f * fstride + (k * ny + j) * pitch + i] with
 *    fstride = pitch * ny * nz (cosmos_field_stride).  Field order:
 *      0 chi, 1..6 gt_xx gt_xy gt_xz gt_yy gt_yz gt_zz, 7 K,
 *      8..13 At_xx..At_zz, 14..16 Gt^x Gt^y Gt^z, 17 alpha,
 *      18..20 beta^x..z, 21..23 B^x..z,
 *      then (fluid on) 24 tau~ = sqrt(gamma) E, 25..27 S~_i = sqrt(gamma) J_i,
 *      then (scalar on) phi, Pi  (Pi = -n^mu d_mu phi).
 *    Padding columns i in [nx, pitch) are never read or written.
 *    Limits: nz <= 65535, ceil(ny / 4) <= 65535 and fstride < 2^31 (one
 *    field's element offsets fit in 32 bits; a state of 24 such fields
 *    would exceed the device memory anyway); else COSMOS_EINVAL.
 *  - Memory: every pointer named state/rhs/ws/... is DEVICE memory owned by
 *    the caller (e.g. a torch CUDA tensor), 16-byte aligned.  The library
 *    allocates no device memory in any call.  Work buffers are passed as
 *    (ws, ws_bytes); cosmos_workspace_bytes gives the size each op needs.
 *  - stream: a cudaStream_t passed as void*; NULL = legacy default stream.
 *    Calls are asynchronous on that stream unless stated otherwise.
 *  - Return value: COSMOS_OK (0) or a negative error code; no call throws.
 *    Arguments are validated before any launch; on error nothing is
 *    launched.  COSMOS_ECUDA reports a failed CUDA launch or copy
 *    (cosmos_last_cuda_error gives the cudaError_t value).
 */
#ifndef COSMOS_GB300_H
#define COSMOS_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define COSMOS_OK 0
#define COSMOS_EINVAL (-1)      /* bad argument (sizes, NULL pointer, option) */
#define COSMOS_ECUDA (-2)       /* CUDA runtime error */
#define COSMOS_EWORKSPACE (-3)  /* workspace smaller than cosmos_workspace_bytes */
#define COSMOS_EALIGN (-4)      /* pointer not 16-byte aligned */
#define COSMOS_ENONFINITE (-5)  /* NaN/Inf or unphysical fluid state detected */
#define COSMOS_EIO (-6)         /* a file could not be opened, read or written */
#define COSMOS_ECHECKPOINT (-7) /* checkpoint of another grid / parameters, or corrupt */

/* Workspace ops for cosmos_workspace_bytes */
#define COSMOS_OP_RHS 0
#define COSMOS_OP_RK4 1
#define COSMOS_OP_CONSTRAINTS 2
#define COSMOS_OP_INIT 3
/* ... and for cosmos_adjoint_workspace_bytes */
#define COSMOS_OP_VJP 4
#define COSMOS_OP_ADJOINT 5
#define COSMOS_OP_INIT_VJP 6
#define COSMOS_OP_DIAG 7
#define COSMOS_OP_SCAN 8

typedef struct {
  int nx, ny, nz; /* grid points per direction, each >= 1 */
  int pitch;      /* doubles between rows (>= nx) */
  double h[3];    /* grid spacing per direction (> 0) */
  double x0[3];   /* coordinates of point (0, 0, 0) */
} cosmos_grid;

typedef struct {
  int slicing;     /* 0: 1+log  d_t alpha = beta.d alpha - 2 alpha (K - K_ref(t));
                      1: harmonic d_t alpha = beta.d alpha - alpha^2 (K - K_ref(t)) */
  int shift;       /* 0: frozen shift (d_t beta = d_t B = 0); 1: Gamma-driver
                      d_t beta = beta.d beta + 3/4 B,
                      d_t B = beta.d B + d_t Gt - beta.d Gt - eta B */
  int fluid;       /* 1: perfect fluid P = w rho (4 extra fields) */
  int scalar;      /* 1: massless scalar field (2 extra fields) */
  double eta;      /* Gamma-driver damping */
  double ko_sigma; /* Kreiss-Oliger strength sigma (>= 0) */
  double w;        /* equation of state P = w rho, 0 < w <= 1 when fluid on */
  double H0, t0;   /* background: K_ref(t) = -3 H0 / (1 + 3/2 (1 + w) H0 (t - t0));
                      H0 = 0 gives K_ref = 0 */
} cosmos_params;

typedef struct {
  int kind;       /* 0: gauge wave  ds^2 = -H dt^2 + H dx^2 + dy^2 + dz^2,
                        H = 1 - A sin(2 pi (x - t)/(nx h_x)), at time t;
                     1: FLRW + curvature perturbation zeta at leading
                        gradient order: gamma_ij = a0^2 e^{2 zeta} delta_ij,
                        K = -3 H0, At = 0, alpha = 1, beta = B = 0, fluid at
                        rest with E fixed by the discrete Hamiltonian
                        constraint (requires fluid on);
                        zeta = mu exp(-r_e^2 / (2 sigma^2)),
                        r_e^2 = sum_i ((x_i - center_i)/q_i)^2;
                     2: kind 1 plus a massless-scalar isocurvature profile
                        (section "Examples", spherically symmetric
                        iso-curvature; the scalar is not part of the
                        background metric): phi = Upsilon = A exp(-r_e^2 /
                        (2 sigma^2)), Pi = 0, and E = (R + 2/3 K^2 -
                        At.At)/(16 pi) - 1/2 chi gt^ij d_i phi d_j phi, so the
                        discrete Hamiltonian constraint with both sources
                        vanishes (requires fluid and scalar on);
                     3: kind 1 at the next-to-leading order of the gradient
                        expansion in eps = k/(aH) (section "Physical system
                        settings", initial-data paragraph: the growing mode
                        up to the next-leading order), constant-mean-
                        curvature slicing, zero shift: with R_ij the Ricci
                        tensor of the leading-order metric (chi0 = a0^-2
                        e^{-2 zeta}, gt = delta), M_ij its trace-free part,
                        delta = chi0 tr R / (6 H0^2):
                        At_ij = 2 chi0 M_ij / ((5 + 3w) H0),
                        gt_ij = delta_ij + h_ij at unit determinant,
                        h_ij = -4 chi0 M_ij / ((5 + 3w)(1 + 3w) H0^2),
                        alpha = 1 - (1 + 3w) delta / (3 (1 + w)),
                        chi = chi0 (1 + 2 delta / (3 (1 + w))), K = -3 H0,
                        Gt^i = gt^jk Gt^i_jk, and the fluid's E and J_i from
                        the discrete Hamiltonian and momentum constraints
                        (requires fluid on and H0 > 0; scalar, if on, zero) */
  double A;
  double mu, sigma;
  double q[3];
  double center[3];
  double a0;
  double t;
} cosmos_id;

/* Number of evolved fields: 24 + 4 fluid + 2 scalar. */
int cosmos_nfields(const cosmos_params* p);

/* Doubles between consecutive fields: pitch * ny * nz. */
size_t cosmos_field_stride(const cosmos_grid* g);

/* Bytes of workspace needed by an op (COSMOS_OP_*); 0 if none. */
size_t cosmos_workspace_bytes(const cosmos_grid* g, const cosmos_params* p, int op);

/* Initial data (section "Physical system settings", initial-data paragraph).
 * Writes every field of `state`.  ws: COSMOS_OP_INIT bytes.  Errors:
 * COSMOS_EINVAL (unknown kind, gauge wave with fluid, kind 2 without fluid
 * and scalar, kind 3 without fluid or with H0 <= 0, sigma, a0 or q not
 * positive), COSMOS_EALIGN, COSMOS_EWORKSPACE. */
int cosmos_init_grid(const cosmos_grid* g, const cosmos_params* p, const cosmos_id* id, double* state, void* ws,
                     size_t ws_bytes, void* stream);

/* Right-hand side d_t U = F(U, t) of every field, written to `rhs` (same
 * layout as state).  Section "Physical system settings": the Einstein
 * equations G = 8 pi T with T = T^SC + T^FL (here in the BSSN chi-form the
 * paper leaves to the textbooks it cites: conformal metric, trace-free
 * extrinsic curvature, K, conformal connection functions, 1+log or harmonic
 * slicing with the background trace K_ref(t), Gamma-driver shift), the
 * matter sources rho_H, J_i, S_ij of the perfect fluid P = w rho and of the
 * massless scalar (box phi = 0), and the fluid's conservation law
 * div T^FL = 0 in conservative 3+1 form with Kurganov-Tadmor face fluxes
 * (same section, last sentence of its first part).  4th-order centred
 * differences; 6th-derivative Kreiss-Oliger dissipation on every field but
 * the fluid's.  ws: COSMOS_OP_RHS bytes.  Errors: COSMOS_EINVAL (grid or
 * parameters, NULL buffer), COSMOS_EALIGN, COSMOS_EWORKSPACE, COSMOS_ECUDA. */
int cosmos_rhs(const cosmos_grid* g, const cosmos_params* p, const double* state, double* rhs, double t, void* ws,
               size_t ws_bytes, void* stream);

/* One fused RK4 stage s in {1, 2, 3, 4} (classic RK4, stage time
 * t + c_s dt with c = 0, 1/2, 1/2, 1):
 *   k = F(U_s, t + c_s dt)
 *   s = 1:  U_next = U_n + dt/2 k,  acc = k
 *   s = 2:  U_next = U_n + dt/2 k,  acc += 2 k
 *   s = 3:  U_next = U_n + dt k,    acc += 2 k
 *   s = 4:  U_n   <- U_n + dt/6 (acc + k)   (U_next unused)
 * U_s must not alias U_next or acc.  U_s = U_n is allowed (stage 1).
 * ws: COSMOS_OP_RHS bytes. */
int cosmos_rk4_stage(const cosmos_grid* g, const cosmos_params* p, int stage, const double* U_s, double* U_n,
                     double* U_next, double* acc, double t, double dt, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * Slab decomposition of one grid over several ranks (one GPU each): every
 * rank holds a slab of z-planes plus 3 ghost planes on each side (the reach
 * of the Kreiss-Oliger stencil), as an ordinary grid of nz_slab + 6 planes.
 * Before each RK4 stage the ranks exchange the ghost planes of the stage
 * state (periodic in z across the ranks) and take the largest of their
 * per-field exponents (cosmos_field_exponents), so that the integer
 * derivative pass rounds exactly as on the whole grid; cosmos_rk4_stage_slab
 * then advances the slab's interior planes.  The results equal the single-
 * grid ones bitwise.  The paper's code runs on one node with OpenMP; this is
 * the GPU form of its grid's natural split.
 * ------------------------------------------------------------------------ */

/* E[s] = the largest biased FP64 exponent over the whole array of limb slot
 * s (slot s = field s; with the fluid on, the scalar's fields move down by 4:
 * 24 + 2 scalar slots), the reference exponent of the integer derivative
 * pass.  E: device memory, 24 + 2 * scalar ints.  Asynchronous. */
int cosmos_field_exponents(const cosmos_grid* g, const cosmos_params* p, const double* state, int* E,
                           void* stream);

/* cosmos_rk4_stage with the algebra pass and the stage combine restricted to
 * planes k_lo .. k_lo + k_cnt - 1 (the derivative and fluid passes cover
 * every plane, so planes within 3 of the range must hold the right values:
 * the ghost planes of a slab), and, if E is not NULL, the derivative pass's
 * reference exponents taken from E (device, as cosmos_field_exponents
 * writes it) instead of its own scan of U_s.  Every entry of E must be at
 * least the exponent cosmos_field_exponents gives for U_s itself (the
 * largest over all ranks is): a smaller one overflows the fixed-point copy
 * and gives wrong derivatives (no fault).  Planes outside the range of U_next
 * / U_n / acc are not written.  ws: COSMOS_OP_RHS bytes.  Errors as
 * cosmos_rk4_stage, and COSMOS_EINVAL for a range outside 0..nz. */
int cosmos_rk4_stage_slab(const cosmos_grid* g, const cosmos_params* p, int stage, const double* U_s, double* U_n,
                          double* U_next, double* acc, double t, double dt, int k_lo, int k_cnt, const int* E,
                          void* ws, size_t ws_bytes, void* stream);

/* One pass of a fused RK4 stage (arguments as cosmos_rk4_stage), so that
 * the passes can be scheduled or timed separately:
 *   pass 0: fluid primitives and face fluxes of U_s (nothing without fluid)
 *   pass 1: derivative pass: finite differences and Kreiss-Oliger terms of U_s
 *   pass 2: algebra pass + stage combine (needs passes 0 and 1 of this stage)
 * Passes 0, 1, 2 in order equal one cosmos_rk4_stage call.  The workspace
 * carries the intermediate results between passes.  Option bits added to
 * `pass` reproduce what cosmos_rk4_step does between its stages:
 *   + 32 (pass 2, stages 1-3): the algebra pass records the largest FP64
 *        exponent of every field it writes to U_next into the workspace
 *        (+ 64: the same, clearing the record first: needed once per
 *        workspace before its first record);
 *   + 16 (pass 1): the derivative pass takes those recorded exponents
 *        instead of scanning U_s, which must then be the U_next of the
 *        recording pass, unchanged since.
 * Results are bitwise those without the options (the same maxima). */
int cosmos_stage_pass(const cosmos_grid* g, const cosmos_params* p, int pass, int stage, const double* U_s,
                      double* U_n, double* U_next, double* acc, double t, double dt, void* ws, size_t ws_bytes,
                      void* stream);

/* One classic RK4 step of size dt from time t of the evolution problem of
 * section "Physical system settings" (the right-hand side of cosmos_rhs),
 * in place on `state`: k_s = F(U_s, t + c_s dt), U_{n+1} = U_n + dt/6
 * (k1 + 2 k2 + 2 k3 + k4), as four cosmos_rk4_stage calls, each fused with
 * its stage combine (stages 2-4 take their fields' largest exponents as the
 * algebra pass of the stage before records them, instead of a scan of the
 * state: bitwise the same).  ws: COSMOS_OP_RK4 bytes (two stage buffers,
 * the accumulator and the fluid buffers).  Errors as cosmos_rhs. */
int cosmos_rk4_step(const cosmos_grid* g, const cosmos_params* p, double* state, double t, double dt, void* ws,
                    size_t ws_bytes, void* stream);

/* cosmos_rk4_step that also keeps the step's stage states: U2 = U_n + dt/2 k1,
 * U3 = U_n + dt/2 k2, U4 = U_n + dt k3 (k_s the right-hand side at stage s),
 * for cosmos_adjoint_step_stages.  U2, U3, U4: caller-owned device buffers in
 * state layout, distinct from state and from each other (else COSMOS_EINVAL).
 * state is updated bitwise as by cosmos_rk4_step.  ws: COSMOS_OP_RK4 bytes. */
int cosmos_rk4_step_stages(const cosmos_grid* g, const cosmos_params* p, double* state, double t, double dt,
                           double* U2, double* U3, double* U4, void* ws, size_t ws_bytes, void* stream);

/* End-to-end step with HOST buffers: copies host_in (pageable or pinned
 * host memory, cosmos_field_stride * nfields doubles, library layout) to
 * dev_state, runs `steps` RK4 steps (ws: COSMOS_OP_RK4 bytes) and copies the
 * result to host_out; synchronous.  host_in and host_out may be the same
 * buffer.  With pinned buffers the copies overlap the computation: the
 * host-to-device copy goes in four field groups on a private stream, each
 * followed by the first derivative pass over those fields, and the
 * device-to-host copy in up to eight slabs of z-planes, each started when the
 * last algebra pass has written them.  The result is bitwise that of
 * cosmos_rk4_step.  Errors: COSMOS_EINVAL (NULL buffer, steps < 0),
 * COSMOS_EALIGN, COSMOS_EWORKSPACE, COSMOS_ECUDA (the call returns only after
 * its own copies have ended, on errors too). */
int cosmos_evolve_host(const cosmos_grid* g, const cosmos_params* p, const double* host_in, double* host_out,
                       double* dev_state, int steps, double t, double dt, void* ws, size_t ws_bytes, void* stream);

/* End-to-end steps of `count` independent states with HOST buffers, pipelined
 * (the RK4 evolution of section "Physical system settings", as cosmos_rk4_step,
 * applied to a sequence of grids, e.g. the states of a parameter scan kept in
 * host memory): state i is copied from host_in[i] to
 * a device buffer, advanced `steps` RK4 steps from time t, and copied back to
 * host_out[i]; every result is bitwise that of cosmos_rk4_step applied
 * `steps` times (and of cosmos_evolve_host).  State i lives in
 * dev_states[i % nbuf] (nbuf caller-owned device buffers of
 * cosmos_field_stride * nfields doubles, 1 <= nbuf <= 16, not overlapping).
 * The copy to the device runs on one private stream, the copy back on
 * another, and the states are advanced in order on `stream`: with pinned
 * host buffers and nbuf >= 2 the copies of the other states overlap each
 * state's computation and each other (pageable buffers give the same
 * results without the overlap).  host_in[i] may repeat (the same inputs
 * evolved again); no host_out[i] may overlap any host_in[j] (COSMOS_EINVAL);
 * host_out entries may repeat (the later state's result is left there).
 * ws: COSMOS_OP_RK4 bytes (unused when steps = 0).  Synchronous: returns when
 * every result is in host memory.  Errors: COSMOS_EINVAL (count or steps < 0,
 * nbuf out of range, a NULL or overlapping buffer), COSMOS_EALIGN,
 * COSMOS_EWORKSPACE, COSMOS_ECUDA (then the contents of the buffers are
 * undefined; the call still returns only after its own copies have ended). */
int cosmos_evolve_host_many(const cosmos_grid* g, const cosmos_params* p, int count, const double* const* host_in,
                            double* const* host_out, double* const* dev_states, int nbuf, int steps, double t,
                            double dt, void* ws, size_t ws_bytes, void* stream);

/* Hamiltonian and (conformal) momentum constraints, the parts of the
 * Einstein equations that the initial data must satisfy (section "Physical
 * system settings", initial-data paragraph: the fluid is generated to meet
 * them, and they hold to rounding precision at the start)
 *   H   = R + 2/3 K^2 - At_ij At^ij - 16 pi rho_H
 *   M^i = gt^ik gt^jl Dt_j At_kl - 3/(2 chi) At^ij d_j chi - 2/3 gt^ij d_j K - 8 pi gt^ij J_j
 * per point into ham_mom (4 fields in state layout, or NULL) and their norms
 * into norms_host[8] = {L2(H), L2(Mx), L2(My), L2(Mz), Linf(H), ...},
 * L2 = sqrt(mean square over all points).  Synchronous (norms on the host).
 * ws: COSMOS_OP_CONSTRAINTS bytes. */
int cosmos_constraints(const cosmos_grid* g, const cosmos_params* p, const double* state, double* ham_mom,
                       double norms_host[8], void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * Reverse mode (adjoint) of the evolution, for gradients of collapse
 * diagnostics with respect to the initial curvature perturbation.  Covers
 * every matter variant (vacuum, fluid, scalar, fluid + scalar); the initial-
 * data maps and the compaction function need the fluid on.  Every reverse
 * step is the exact transpose
 * of the corresponding discrete forward step (minmod, max and |.| take the
 * derivative of the branch taken).
 * ------------------------------------------------------------------------ */

/* Workspace for COSMOS_OP_VJP, COSMOS_OP_ADJOINT, COSMOS_OP_INIT_VJP or
 * COSMOS_OP_DIAG (0 if the arguments are invalid). */
size_t cosmos_adjoint_workspace_bytes(const cosmos_grid* g, const cosmos_params* p, int op);

/* v = (dF/dU)^T w: the transpose of the right-hand side's Jacobian at state
 * U and time t applied to w (both in state layout).  v is overwritten. */
int cosmos_rhs_vjp(const cosmos_grid* g, const cosmos_params* p, const double* U, const double* w, double* v,
                   double t, void* ws, size_t ws_bytes, void* stream);

/* Adjoint of one RK4 step U_{n+1} = Phi(U_n) of cosmos_rk4_step from time t
 * with step dt: lam_n = (dPhi/dU_n)^T lam_np1, stage by stage in reverse
 * (the paper has no adjoint: this serves gradients of the collapse
 * diagnostics of its PBH examples, section "Examples", with respect to the
 * initial curvature perturbation of its initial-data paragraph).
 * Recomputes the stage states from U_n.  lam_n may equal lam_np1 (in
 * place).  ws: COSMOS_OP_ADJOINT bytes.  Errors as cosmos_rhs. */
int cosmos_adjoint_step(const cosmos_grid* g, const cosmos_params* p, const double* U_n, const double* lam_np1,
                        double* lam_n, double t, double dt, void* ws, size_t ws_bytes, void* stream);

/* cosmos_adjoint_step with the step's stage states U2, U3, U4 supplied (as
 * written by cosmos_rk4_step_stages from U_n at the same t, dt) instead of
 * recomputed: three forward stages fewer per step, the same result bitwise.
 * lam_n may equal lam_np1; it must not alias a state.  ws: COSMOS_OP_ADJOINT
 * bytes. */
int cosmos_adjoint_step_stages(const cosmos_grid* g, const cosmos_params* p, const double* U_n, const double* U2,
                               const double* U3, const double* U4, const double* lam_np1, double* lam_n, double t,
                               double dt, void* ws, size_t ws_bytes, void* stream);

/* FLRW initial data (as cosmos_init_grid kind 1) from a per-point curvature
 * perturbation zeta (one double per point, state row layout):
 * chi = exp(-2 zeta)/a0^2, gt = delta, K = -3 H0, alpha = 1, fluid at rest
 * with E from the discrete Hamiltonian constraint.  ws: COSMOS_OP_INIT bytes. */
int cosmos_init_zeta(const cosmos_grid* g, const cosmos_params* p, const double* zeta, double a0, double* state,
                     void* ws, size_t ws_bytes, void* stream);

/* zeta_bar = (d state0 / d zeta)^T lam0 for the map of cosmos_init_zeta
 * (state0 = its output).  ws: COSMOS_OP_INIT_VJP bytes. */
int cosmos_init_zeta_vjp(const cosmos_grid* g, const cosmos_params* p, const double* state0, const double* lam0,
                         double* zeta_bar, void* ws, size_t ws_bytes, void* stream);

/* Compaction function about the centre grid point (nx/2, ny/2, nz/2), fluid on:
 *   C(r_k) = 2 dM(r_k) / R(r_k),  r_k = k h,  k = 1..kmax (kmax < min(n)/2),
 *   dM = h^3 sum_{|x - c| < r_k} (tau~ - Ebar sqrt(gamma)),  Ebar = sum tau~ / sum sqrt(gamma),
 *   R = r_k * mean of chi^{-1/2} over the 6 axis points at distance r_k.
 * Writes C_host[k-1] and aux_host[4 kmax + 2] (per k: S, V, R, dM; then the
 * box sums of tau~ and sqrt(gamma)) for cosmos_compaction_vjp.  Sums run in a
 * fixed order (deterministic).  Synchronous.  ws: COSMOS_OP_DIAG bytes. */
int cosmos_compaction(const cosmos_grid* g, const cosmos_params* p, const double* state, double* C_host, int kmax,
                      double* aux_host, void* ws, size_t ws_bytes, void* stream);

/* lam = cbar * d C(r_kstar) / d state (state layout, overwritten), with the
 * aux_host written by cosmos_compaction for the same state. */
int cosmos_compaction_vjp(const cosmos_grid* g, const cosmos_params* p, const double* state, int kstar, int kmax,
                          const double* aux_host, double cbar, double* lam, void* stream);

/* Central lapse of a run (the collapse diagnostic the paper's PBH examples
 * follow, section "Examples": the lapse at the centre of the overdensity
 * falls as it collapses).  Copies alpha at the centre grid point
 * (nx/2, ny/2, nz/2) of `state` into series[index] (device memory, at least
 * index + 1 doubles).  Asynchronous.  Errors: COSMOS_EINVAL. */
int cosmos_central_lapse(const cosmos_grid* g, const cosmos_params* p, const double* state, double* series,
                         int index, void* stream);

/* Reverse of cosmos_central_lapse: lam[alpha at the centre point] += abar
 * (lam in state layout, device).  Asynchronous. */
int cosmos_central_lapse_vjp(const cosmos_grid* g, const cosmos_params* p, double abar, double* lam, void* stream);

/* Minimum of series[0 .. count-1] (device) and the first index attaining
 * it: result[0] = the minimum, result[1] = its index as a double (device,
 * 2 doubles).  One warp scans in a fixed order (deterministic); a NaN
 * entry never wins against a number.  Asynchronous.  Errors: COSMOS_EINVAL
 * (NULL pointer, count < 1). */
int cosmos_series_argmin(const double* series, int count, double* result, void* stream);

/* ------------------------------------------------------------------------
 * Batched evolution of many independent grids (a threshold scan: one
 * instance per amplitude or shape of the initial perturbation, grids of
 * uneven sizes, each with its own dt).  All instances share one
 * cosmos_params.  Per RK4 stage, one persistent launch (plus the two fluid
 * passes when the fluid is on) sweeps a flat work list holding every point
 * of every instance, so small or uneven grids leave no SM idle; a run of
 * several steps can be captured once into a CUDA graph and replayed.
 * ------------------------------------------------------------------------ */
typedef struct cosmos_batch_s* cosmos_batch;

typedef struct {
  int mapping;       /* 0: 2D tiles of block_x x block_y points in one z-plane;
                        1: runs of block_x * block_y consecutive points */
  int block_x, block_y; /* block_x * block_y must be 128 */
  int blocks_per_sm; /* persistent grid = blocks_per_sm * SM count, 1..3 */
} cosmos_batch_tuning;

/* Device workspace for a batch: per instance two stage buffers, the RK4
 * accumulator and the fluid buffers, plus the work list and the per-step
 * K_ref table for up to max_steps steps. */
size_t cosmos_batch_workspace_bytes(int n, const cosmos_grid* grids, const cosmos_params* p, int max_steps);

/* Build a plan (host memory, freed by cosmos_batch_free) over n instances:
 * grids[i], time step dt[i], start time t0[i] and device state states[i]
 * (layout of include/cosmos.h).  Copies the work list and tables into `ws`
 * (synchronous).  tuning = NULL picks 2D tiles 32 x 4, 3 blocks per SM. */
int cosmos_batch_plan(int n, const cosmos_grid* grids, const cosmos_params* p, const double* dt, const double* t0,
                      double* const* states, int max_steps, const cosmos_batch_tuning* tuning, void* ws,
                      size_t ws_bytes, cosmos_batch* plan_out);

/* Change the work-list mapping / launch shape (synchronous; drops any
 * captured graph). */
int cosmos_batch_set_tuning(cosmos_batch plan, const cosmos_batch_tuning* tuning);

/* Advance every instance by `steps` RK4 steps, global step indices
 * first_step .. first_step + steps - 1 (<= max_steps).  use_graph = 1
 * captures the whole sequence into a CUDA graph on the first call with these
 * (first_step, steps) and replays it afterwards; it needs a non-NULL stream.
 * Asynchronous on `stream`. */
int cosmos_batch_run(cosmos_batch plan, int first_step, int steps, int use_graph, void* stream);

/* Mean time of one RK4 stage-1 pass over the whole batch with the current
 * tuning, over `reps` passes, in milliseconds (CUDA events; synchronous).
 * Stage 1 writes only the stage buffers and accumulators, so the instance
 * states are unchanged.  Used by the autotuner. */
int cosmos_batch_time_stage(cosmos_batch plan, int reps, double* ms_out, void* stream);

/* The built-in candidate tunings of the autotuner: copies up to `max` of
 * them into `out` (may be NULL) and returns how many there are.  Host only. */
int cosmos_batch_default_candidates(cosmos_batch_tuning* out, int max);

/* Autotuner: times every candidate tuning with cosmos_batch_time_stage
 * (`reps` passes each, after one warm-up pass) and leaves the fastest set in
 * the plan.  candidates = NULL with n_candidates = 0 takes the built-in list.
 * cache_path (may be NULL): a text file with one line per key, the key being
 * the device name, the matter model and every grid size in order.  A line for
 * this plan's key sets its tuning without timing anything (*cache_hit = 1,
 * ms_out filled with NaN); otherwise the search runs and the line is written
 * (the file is rewritten through a temporary copy renamed over it).
 * best_out (may be NULL): the chosen tuning; ms_out (n entries or NULL): the
 * mean stage time of each candidate in ms.  Synchronous; the instance states
 * are unchanged.  Errors: COSMOS_EINVAL (NULL plan, reps < 1, an invalid
 * candidate), COSMOS_ECUDA, COSMOS_EIO (cache not written; the tuning is set). */
int cosmos_batch_autotune(cosmos_batch plan, const cosmos_batch_tuning* candidates, int n_candidates, int reps,
                          const char* cache_path, cosmos_batch_tuning* best_out, double* ms_out, int* cache_hit,
                          void* stream);

void cosmos_batch_free(cosmos_batch plan);

/* ------------------------------------------------------------------------
 * Fixed mesh refinement (section "Statement of need": nested refinement
 * levels resolve the collapsing region; the paper's figure of the lapse at
 * horizon formation shows the lowest level and two refined ones).  The paper
 * gives no scheme; this one:
 *  - level 0 is the periodic box grid[0]; level l >= 1 is one box grid[l]
 *    with h = h_{l-1}/2 (exactly) and x0 = x0_{l-1} + origin[l] * h, so that
 *    every other point of level l lies on a point of level l-1;
 *  - along each axis, level l is either a box with interior [lo, hi),
 *    lo >= 3 and n - hi >= 3 ghost layers, or, where level l-1 is periodic,
 *    periodic too (lo = 0, hi = n = 2 n_{l-1}, origin = 0);
 *  - ghost points are set before every RK4 stage from level l-1: in time from
 *    the continuous extension of order 3 of the parent's RK4 step, in the
 *    stage-consistent form (the stage states RK4 forms from the solution's
 *    Taylor expansion at the substep's start); in space by the tensor product
 *    of 6-point Lagrange interpolation at half-way points and injection at
 *    coincident points.  The parent points these read must lie in the
 *    parent's interior (or wrap on a periodic parent axis), else EINVAL;
 *  - Berger-Oliger subcycling: level l takes two steps of dt_{l-1}/2 after
 *    each step of level l-1, then its interior points that lie on level l-1
 *    points overwrite those (injection);
 *  - after a hierarchy step every level's ghost points hold the values
 *    interpolated from its parent's new state.
 * States use the layout of cosmos_grid for each level (ghost points
 * included); the right-hand side is exact at interior points only.
 * ------------------------------------------------------------------------ */
#define COSMOS_FMR_MAX_LEVELS 8

typedef struct {
  int levels;                                  /* 1 .. COSMOS_FMR_MAX_LEVELS */
  cosmos_grid grid[COSMOS_FMR_MAX_LEVELS];     /* per level */
  int origin[COSMOS_FMR_MAX_LEVELS][3];        /* level l >= 1 (level 0 ignored) */
  int lo[COSMOS_FMR_MAX_LEVELS][3];            /* interior [lo, hi) of level l >= 1 */
  int hi[COSMOS_FMR_MAX_LEVELS][3];
} cosmos_fmr;

/* Device workspace of the hierarchy calls: one RK4 workspace for the largest
 * level, the four saved states (U_n and the three stage states) of every
 * level that has a finer one, and the interpolation buffer.  0 if the
 * hierarchy is invalid. */
size_t cosmos_fmr_workspace_bytes(const cosmos_fmr* m, const cosmos_params* p);

/* Initial data (cosmos_init_grid on every level, the gauge wave's wavelength
 * being level 0's box), injection from the finest level down, then the ghost
 * points of every level from its parent.  states[l]: level l's device state. */
int cosmos_fmr_init(const cosmos_fmr* m, const cosmos_params* p, const cosmos_id* id, double* const* states,
                    void* ws, size_t ws_bytes, void* stream);

/* One step of the hierarchy from time t: level l takes 2^l RK4 steps of
 * dt0 / 2^l (Berger-Oliger order).  Asynchronous on `stream`.  Errors:
 * COSMOS_EINVAL (hierarchy, NULL or repeated state, dt0 <= 0), COSMOS_EALIGN,
 * COSMOS_EWORKSPACE, COSMOS_ECUDA. */
int cosmos_fmr_step(const cosmos_fmr* m, const cosmos_params* p, double* const* states, double t, double dt0,
                    void* ws, size_t ws_bytes, void* stream);

/* Ghost points of level `level` (>= 1) of `child` from the parent state
 * `parent` (spatial interpolation only); interior points are not touched. */
int cosmos_fmr_prolong(const cosmos_fmr* m, const cosmos_params* p, int level, const double* parent, double* child,
                       void* ws, size_t ws_bytes, void* stream);

/* Injection: the interior points of level `level` (>= 1) that lie on points of
 * its parent overwrite those values of `parent`. */
int cosmos_fmr_restrict(const cosmos_fmr* m, const cosmos_params* p, int level, const double* child, double* parent,
                        void* stream);

/* cosmos_constraints without a workspace argument, for callers that cannot
 * allocate device memory while they run: a host application whose device
 * memory is handed out by its own pool or framework, which forbids
 * cudaMalloc/cudaFree once it is running (they can synchronise the whole
 * device and stall its other streams), or a monitoring hook that must not
 * change the process's memory footprint.  The paper has no counterpart; this
 * is a library-usage variant of cosmos_constraints with the same outputs and
 * the same synchronous behaviour: it copies the norms to the host and
 * synchronises `stream` before it returns.
 *
 * Scratch: one static device array of 2^21 doubles (16 MiB) inside the
 * library, which every GPU that loads the library keeps until the process
 * exits.  It must hold (fluid on: 4 * cosmos_field_stride, rounded up to 32
 * doubles) + 8 * (number of 32 x 4 thread blocks over the grid, rounded up to
 * 32) + 8 doubles; larger grids return COSMOS_EWORKSPACE before anything is
 * launched (e.g. 256^3 vacuum fits; with the fluid on, up to about 80^3).
 * The first call made with a device current resolves the array's device
 * address for that device (cudaGetSymbolAddress) and keeps it for the rest
 * of the process.  The call cannot run under stream capture: it copies the
 * norms to the host and synchronises `stream`.  After a
 * cudaDeviceReset the kept address may no longer be valid: this call is not
 * for processes that reset a device they have used it on.  The call
 * allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 * Arguments are checked as cosmos_constraints checks them.
 * Every call overwrites all the scratch it reads, so no state carries over
 * between calls, but all calls share the one array: calls that can overlap
 * on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  On COSMOS_ECUDA the CUDA runtime's
 * cudaGetLastError() gives the error. */
int cosmos_constraints_noalloc(const cosmos_grid* g, const cosmos_params* p, const double* state, double* ham_mom,
                               double norms_host[8], void* stream);

/* Failure detection: counts, per field, the values of `state` that are NaN
 * or Inf and, with the fluid on, the points where tau~ <= 0 (no fluid state
 * has a non-positive energy density, so the primitive recovery has no
 * solution there).  A reduction over the grid, never a trap; padding
 * columns are not read.  counts_host: cosmos_nfields(p) ints, or NULL.
 * Synchronous.  Returns COSMOS_OK when nothing was found,
 * COSMOS_ENONFINITE when something was, else EINVAL / EALIGN / EWORKSPACE /
 * ECUDA.  ws: COSMOS_OP_SCAN bytes. */
int cosmos_scan_state(const cosmos_grid* g, const cosmos_params* p, const double* state, int* counts_host, void* ws,
                      size_t ws_bytes, void* stream);

/* Measured FP64 fused-multiply-add throughput of the current device, in
 * flop/s (2 flop per DFMA), from a timed launch of independent DFMA chains
 * on every SM.  Synchronous; allocates nothing (writes one double per thread
 * into `scratch`, which must hold 152 * 8 * 256 doubles). */
int cosmos_probe_fp64(double* scratch, double* flops_out, void* stream);

/* cudaError_t of the last COSMOS_ECUDA returned by this thread. */
int cosmos_last_cuda_error(void);

/* ------------------------------------------------------------------------
 * Checkpoint / resume of one grid's state.  File: a 4096-byte text header
 * (one JSON object, padded with spaces, ending in a newline: "format"
 * "cosmos-checkpoint", "version" 1, "byte_order", "n" [nx, ny, nz], "h",
 * "x0", "nfields", "fields" (names in state order), "params" (slicing, shift,
 * fluid, scalar, eta, ko_sigma, w, H0, t0), "t", "step", "payload_bytes",
 * "payload_fnv1a64" (hex)), then every field as nx * ny * nz binary64 values,
 * i fastest, field after field (padding columns not stored).  Doubles in the
 * header carry 17 significant digits, so they read back exactly.
 * state_on_device: 1 for a device buffer (copied through host memory on
 * `stream`, synchronously), 0 for a host buffer of the same pitched layout.
 * ------------------------------------------------------------------------ */

/* Writes `path` through a temporary file "<path>.partial" renamed over it.
 * Errors: COSMOS_EINVAL, COSMOS_EIO, COSMOS_ECUDA. */
int cosmos_checkpoint_save(const char* path, const cosmos_grid* g, const cosmos_params* p, const double* state,
                           int state_on_device, double t, long long step, void* stream);

/* Reads `path` into `state` and returns its time and step counter.  The
 * header must give exactly this grid (sizes, spacing, origin) and these
 * parameters, and the payload must have the stated size and hash, else
 * COSMOS_ECHECKPOINT and `state` is not written (a first pass over the file
 * checks all of this; a second pass copies the payload in, hashing it again).
 * COSMOS_EIO: the file failed to read, or changed, during the second pass;
 * `state` then holds part of the file or unverified data and must not be
 * used.  Errors also COSMOS_EINVAL, COSMOS_ECUDA. */
int cosmos_checkpoint_load(const char* path, const cosmos_grid* g, const cosmos_params* p, double* state,
                           int state_on_device, double* t_out, long long* step_out, void* stream);

/* Static description of an error code. */
const char* cosmos_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* COSMOS_GB300_H */
