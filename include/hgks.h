/*
 * hgks.h -- C ABI of the GB300 (sm_103a) implementation of the high-order
 * gas-kinetic scheme with third-order 3D WENO-AO reconstruction of Pan & Xu,
 * "High-order gas-kinetic scheme with three-dimensional WENO reconstruction
 * for the Euler and Navier-Stokes solutions" (arXiv 1909.01580).
 *
 * Conventions shared by every entry point:
 *   - Every call returns an int status (HGKS_OK or a negative HGKS_E_* code);
 *     nothing crosses the ABI as an exception.  hgks_last_error() gives a
 *     one-line reason for the last failure on a handle.
 *   - A handle owns all of its device memory; the caller owns every host
 *     buffer it passes.  Buffers flagged on_device = 1 are device pointers
 *     on the handle's device, valid in stream order on the handle's stream.
 *   - State arrays are conservative cell averages (rho, rho U, rho V, rho W,
 *     rho E) in SoA layout [5][nz][ny][nx], x fastest, FP64.
 *   - Calls are ordered on the handle's stream.  Calls that return host
 *     data or a status synchronise that stream before returning.
 *   - There is no CPU fallback: without a usable CUDA device hgks_create
 *     fails with HGKS_E_CUDA.
 */
#ifndef HGKS_H
#define HGKS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hgks hgks_t;

/* Mesh and arithmetic of a solver instance. */
typedef struct {
    int n[3];          /* cells in x, y, z (x fastest in memory)                    */
    double lo[3];      /* physical box [lo, hi]                                     */
    double hi[3];
    int mesh;          /* 0: uniform mesh of cubic cells (Sec. 4 accuracy, TGV and
                             Riemann tests);
                          1: static mapped mesh of trilinear hexahedra (Sec. 2,
                             Sec. 4 non-coplanar mesh), x_d = xi_d + amp
                             prod_e sin(2 pi (xi_e - lo_e)/L_e) on a uniform
                             reference grid xi over [lo, hi];
                          2: the same map times sin(omega t), moving with the
                             grid velocity dx/dt (Remark 2).
                          Mapped meshes are periodic in every direction.      */
    double mesh_amp;   /* amp of the map (0 for mesh 0)                             */
    double mesh_omega; /* omega of the moving map (0 for meshes 0 and 1)            */
    int precision;     /* HGKS_FP64 or HGKS_MIXED                                   */
} hgks_grid_t;

enum { HGKS_FP64 = 0,   /* every operation in FP64                               */
       HGKS_MIXED = 1   /* reconstruction and Gauss-point flux in FP32; face-flux
                           accumulation and the two-stage update in FP64         */
};

enum { HGKS_BC_PERIODIC = 0, HGKS_BC_REFLECTIVE = 1, HGKS_BC_OUTFLOW = 2 };

/* Largest number of cells along one axis (index arithmetic on the device is
 * 32-bit); larger grids give HGKS_E_INVALID. */
#define HGKS_MAX_CELLS_PER_AXIS 1024

enum {
    HGKS_OK = 0,
    HGKS_E_INVALID = -1,     /* bad argument                                     */
    HGKS_E_NOMEM = -2,       /* device allocation failed                         */
    HGKS_E_CUDA = -3,        /* CUDA runtime error                               */
    HGKS_E_NONPHYSICAL = -4, /* NaN or non-positive density/pressure after a step */
    HGKS_E_TIMEOUT = -5,     /* a bounded device wait gave up                    */
    HGKS_E_STATE = -6        /* call out of order (e.g. step before set_state)   */
};

/* Create a solver on the current CUDA device.
 *   grid    mesh and precision (see hgks_grid_t); cells must be cubes and
 *           every axis needs at least 2 cells (3 on an axis with a reflective side).
 *   gamma   ratio of specific heats; K = (5 - 3 gamma)/(gamma - 1) internal
 *           degrees of freedom of the Maxwellian (Sec. 3, BGK model).
 *   mu      dynamic viscosity.  mu = 0 selects the inviscid collision time
 *           tau = eps dt + C |p_l - p_r|/(p_l + p_r) dt, mu > 0 the viscous one
 *           tau = mu/p + C |p_l - p_r|/(p_l + p_r) dt (Sec. 4).
 *   Pr      Prandtl number; when mu > 0 and Pr != 1 the energy flux takes the
 *           heat-flux correction F_E += (1/Pr - 1) q (the paper is silent on
 *           Pr; this is the usual BGK correction).
 *   bc      per face -x,+x,-y,+y,-z,+z: HGKS_BC_PERIODIC (must pair),
 *           HGKS_BC_REFLECTIVE (mirror, normal momentum negated) or
 *           HGKS_BC_OUTFLOW (the non-reflecting boundary of the Riemann
 *           problems of Sec. 4, read as zero-gradient extrapolation: every
 *           ghost layer repeats the boundary cell).
 *   stream  cudaStream_t to order all work on, or NULL for a private stream.
 *   out     receives the handle.
 * Paper constants are defaults: Gamma = 0.0025 (gamma_0 = 0.94), epsilon
 * = 1e-8 in the nonlinear weights, tau constants eps = 0.01, C = 1;
 * hgks_set_option changes them. */
int hgks_create(const hgks_grid_t *grid, double gamma, double mu, double Pr, const int bc[6], void *stream,
                hgks_t **out);

/* Change a scheme constant: "Gamma" (linear weight of each of the 24
 * sub-stencils, Sec. 2), "weno_eps", "weno_pow" (1 or 2, exponent of
 * tau/(beta + eps) in eq. nonlinear), "tau_eps", "tau_C" (collision time,
 * Sec. 4), "limiter" (1/0: positivity fallback of Sec. 4), "mu_power" and
 * "mu_T_ref" (viscosity law mu (T/T_ref)^mu_power of the isotropic
 * turbulence of Sec. 4, 0.76 there, evaluated at the temperature p/rho of
 * the interface equilibrium state in the collision time; mu_power = 0, the
 * default, keeps mu constant), "stencil" (0: the big stencil S with its
 * 24 sub-stencils; 1: S' of the Remark of Sec. 2, S plus the six axis cells
 * two steps away, with the 8 octant sub-stencils and gamma_0 = 1 - 8 Gamma;
 * uniform mesh and conservative variables only), "characteristic" (1/0:
 * reconstruct the
 * characteristic variables L Q of
 * Sec. 4, L the inverse of the right eigenvectors of the Euler flux
 * Jacobian along the face normal at the mean of the face's two cell
 * averages; both sides of every face are reconstructed in that basis, so
 * the reconstruction costs about six times the conservative one and the
 * handle allocates 2 x 50 values per face in the working precision;
 * uniform mesh only, HGKS_E_INVALID otherwise; hgks_reconstruct then
 * returns HGKS_E_STATE, the polynomials being per face and side).
 * Returns HGKS_E_INVALID for an unknown key or value, HGKS_E_NOMEM when
 * the characteristic buffers cannot be allocated. */
int hgks_set_option(hgks_t *h, const char *key, double value);

/* Load the state q ([5][nz][ny][nx] FP64, copied) at time t.  on_device: 1
 * when q is device memory (ordered on the handle's stream, no
 * synchronisation), 0 for host memory (the call returns once q has been
 * read).  Host memory that the GPU can address (pinned or registered:
 * cudaHostAlloc, cudaHostRegister) is read by the kernel that lays the state
 * out, over the host link; other host memory is copied to a device buffer
 * first.  On a mapped
 * mesh the cell volumes that the update divides by restart from the
 * geometric volumes of the mesh at t.  On a moving mesh each step freezes
 * the geometry at the start of each stage (t_n, then t_n + dt/2), takes the
 * flux in the frame moving with the grid, advances |Omega| Q by the two-stage
 * formula and the volume by the same formula from the swept-volume rate of
 * the faces (discrete geometric conservation: a uniform flow stays uniform). */
int hgks_set_state(hgks_t *h, const double *q, int on_device, double t);

/* Copy the state out into q ([5][nz][ny][nx] FP64) and the time into *t
 * (t may be NULL).  on_device as for hgks_set_state: host memory that the
 * GPU can address is written by the kernel that gathers the interior, other
 * host memory through a device buffer; with host memory (or t) the call
 * returns once q (and *t) hold the state. */
int hgks_get_state(hgks_t *h, double *q, int on_device, double *t);

/* Advance nsteps two-stage fourth-order steps (Sec. 3):
 *   Q*      = Q^n + dt/2 L(Q^n) + dt^2/8 dL/dt(Q^n)
 *   Q^{n+1} = Q^n + dt L(Q^n) + dt^2/6 (dL/dt(Q^n) + 2 dL/dt(Q*)).
 * dt_fixed > 0 fixes dt; otherwise dt = cfl * min_cells h/(|U| + c),
 * reduced on the device and clipped so that t does not pass t_end; steps
 * after t reaches t_end do nothing (with a finite t_end the call checks every
 * 16 steps and stops issuing them).  *t_out and *steps_done (either may be
 * NULL) receive the time reached and the steps taken; passing them
 * synchronises the stream.  Returns HGKS_E_NONPHYSICAL if a step produced
 * NaN or non-positive density or pressure. */
int hgks_step(hgks_t *h, int nsteps, double cfl, double dt_fixed, double t_end, double *t_out, int *steps_done);

/* The finite-volume operator L(Q) = -1/|Omega| sum_faces F.n (eq. finite)
 * and its time derivative dL/dt(Q) for the resident state with time step
 * dt (which enters the flux through the collision time and the two time
 * levels dt, dt/2 of eq. expansion-1).  L and dLdt: [5][nz][ny][nx] FP64. */
int hgks_flux(hgks_t *h, double dt, double *L, double *dLdt, int on_device);

/* The reconstructed polynomial of every interior cell (Sec. 2): coef
 * [ncell][5][9] FP64 (always FP64 on output) holds the coefficients of
 * P~ = Q_c + sum_n c_n p_n in the scaled coordinates X = (x - x_c)/h, with
 * p_n = (X, Y, Z, X^2 - 1/12, Y^2 - 1/12, Z^2 - 1/12, XY, XZ, YZ); flag
 * [ncell] int (may be NULL) is 1 where the positivity fallback set P~ = Q_c.
 * Host buffers. */
int hgks_reconstruct(hgks_t *h, double *coef, int *flag);

/* Gas-kinetic flux at n Gauss points (Sec. 3, eq. flux with the time
 * integrals of eq. expansion-1), a test surface for the flux kernel.
 *   in     [n][40] FP64 host, local frame (n_x, n_y, n_z), n_x from the left
 *          to the right cell: W_l, dW_l/dn_x, dW_l/dn_y, dW_l/dn_z, W_r,
 *          dW_r/dn_x, dW_r/dn_y, dW_r/dn_z (5 values each).
 *   ug     [n][3] grid velocity in the local frame, or NULL for a fixed mesh.
 *   dt     time step.
 *   params gamma, mu, Pr, tau_eps, tau_C.
 *   precision HGKS_FP64 or HGKS_MIXED (FP32 arithmetic).
 *   F, dF  [n][5] FP64 host outputs: flux per unit area and its time
 *          derivative in the local frame. */
int hgks_point_flux(int n, const double *in, const double *ug, double dt, const double params[5], int precision,
                    double *F, double *dF);

/* Phases of a stage, for hgks_get_timing. */
enum { HGKS_PHASE_HALO = 0,   /* ghost fill                                 */
       HGKS_PHASE_RECON = 1,  /* WENO-AO reconstruction (Sec. 2)            */
       HGKS_PHASE_FLUX = 2,   /* Gauss-point gas-kinetic face flux (Sec. 3) */
       HGKS_PHASE_UPDATE = 3, /* two-stage update (Sec. 3)                  */
       HGKS_PHASE_CFL = 4,    /* CFL reduction and dt                        */
       HGKS_NPHASE = 5 };

/* Turn per-phase timing on (1) or off (0) and reset the accumulators.  While
 * on, each launch group of a phase is bracketed by CUDA events recorded on
 * the handle's stream.  Synchronises the stream. */
int hgks_set_timing(hgks_t *h, int enable);

/* Device time (ms, CUDA events) and kernel launches accumulated per phase
 * since the last hgks_set_timing.  ms and launches: [HGKS_NPHASE] host
 * arrays.  Synchronises the stream. */
int hgks_get_timing(hgks_t *h, double ms[HGKS_NPHASE], unsigned long long launches[HGKS_NPHASE]);

/* ---------------------------------------------------------------------------
 * Batched execution (system layer around the paper's method; the paper has
 * no counterpart).  Many instances of different grid sizes and flow
 * parameters advance together: each phase of a stage (CFL reduction, ghost
 * fill, reconstruction, the three face-flux directions, update) is one
 * persistent launch over a tile table that spans every resident instance,
 * and a whole step is one CUDA graph launch.  Each instance takes its own dt
 * from its own CFL reduction and stops at its own end time; an instance's
 * arithmetic is the same alone and in a batch.  Instances live in one device
 * arena allocated at creation: adding and removing them allocates nothing
 * on the device.
 * ------------------------------------------------------------------------- */
typedef struct hgks_batch hgks_batch_t;

/* Number of tuning parameters: [0] tile schedule (0 slot order, 1 largest
 * instance first, 2 round robin), [1..5] tile size in multiples of the
 * block for the CFL, ghost, reconstruction, flux and update phases,
 * [6..10] persistent blocks per SM for the same phases. */
#define HGKS_TUNE_NPARAM 11

/* Create a batch of at most max_instances instances with arena_bytes of
 * device memory for them (one allocation, here), all in one precision. */
int hgks_batch_create(int precision, unsigned long long arena_bytes, int max_instances, void *stream,
                      hgks_batch_t **out);

/* Arena bytes one instance of this grid needs (0 for an invalid grid):
 * the admission test of a serving loop. */
unsigned long long hgks_batch_footprint(const hgks_grid_t *grid);

/* Admit an instance: grid/gamma/mu/Pr/bc as for hgks_create (grid->precision
 * must equal the batch's), q its initial state ([5][nz][ny][nx] FP64 host),
 * t0 its time, t_end its end time, cfl its CFL number.  *slot receives its
 * slot.  HGKS_E_NOMEM when no slot or not enough free arena is left;
 * HGKS_E_NONPHYSICAL (nothing admitted, the resident instances untouched)
 * when q holds a non-finite value or a cell with non-positive density or
 * pressure.  Synchronises the batch stream. */
int hgks_batch_add(hgks_batch_t *b, const hgks_grid_t *grid, double gamma, double mu, double Pr, const int bc[6],
                   const double *q, double t0, double t_end, double cfl, int *slot);

/* Retire the instance in slot and return its arena memory. */
int hgks_batch_remove(hgks_batch_t *b, int slot);

/* Advance every resident instance nsteps two-stage steps (instances at
 * their end time do nothing).  Asynchronous: graph launches on the stream. */
int hgks_batch_step(hgks_batch_t *b, int nsteps);

/* Per slot (arrays of max_instances, any may be NULL): time, steps taken,
 * state 0 free, 1 running, 2 reached its end time, 3 nonphysical.
 * Synchronises the batch stream. */
int hgks_batch_poll(hgks_batch_t *b, double *t, int *steps, int *state);

/* Copy the state of the instance in slot to q ([5][nz][ny][nx] FP64 host). */
int hgks_batch_get_state(hgks_batch_t *b, int slot, double *q);

/* Autotuner: coordinate search over the tuning parameters, timing
 * steps_per_trial graph-launched steps of the current batch per candidate
 * (this advances the resident instances), keeps the fastest and returns it
 * in params_out (may be NULL). */
int hgks_batch_tune(hgks_batch_t *b, int steps_per_trial, int params_out[HGKS_TUNE_NPARAM]);

/* Set or read the tuning parameters (see HGKS_TUNE_NPARAM). */
int hgks_batch_set_tuning(hgks_batch_t *b, const int params[HGKS_TUNE_NPARAM]);
int hgks_batch_get_tuning(const hgks_batch_t *b, int params[HGKS_TUNE_NPARAM]);

/* Kernel launches issued by the batch (graph nodes counted per step). */
unsigned long long hgks_batch_launch_count(const hgks_batch_t *b);

/* One-line reason for the last failure on b (or on creation when NULL). */
const char *hgks_batch_last_error(const hgks_batch_t *b);

void hgks_batch_destroy(hgks_batch_t *b);

/* Bytes of device scratch that hgks_flux_noalloc works in (16 MiB). */
#define HGKS_NOALLOC_SCRATCH_BYTES (16 * 1024 * 1024)

/* Allocation-free evaluation of L(Q) and dL/dt(Q), for callers that cannot
 * call cudaMalloc: a serving loop that must not block on the implicit device
 * synchronisation of an allocation, code that lives inside another
 * framework's memory pool, or code under a no-allocation policy after
 * start-up.  The paper has no counterpart; it computes exactly what
 * hgks_flux computes (same kernels, the paper's default constants) without a
 * handle and without allocating: no cudaMalloc, cudaFree or allocating
 * library call.
 *   grid, gamma, mu, Pr, bc  as for hgks_create.
 *   q      device pointer, the state [5][nz][ny][nx] FP64 (read only).
 *   dt     time step, a positive finite number (else HGKS_E_INVALID).
 *   L, dLdt  device pointers [5][nz][ny][nx] FP64 (written).
 *   stream cudaStream_t (or NULL for the legacy default stream); the call is
 *          ordered on it and returns without synchronising.
 * Working memory is one file-scope device array of HGKS_NOALLOC_SCRATCH_BYTES
 * that every GPU loading the library holds until the process exits.  The
 * grid's padded state, reconstruction coefficients and face fluxes must fit
 * in it (mixed: also the split state): cubes of up to 27^3 cells in FP64 and 29^3 mixed; larger
 * grids return HGKS_E_INVALID with the byte count in hgks_last_error(NULL).
 * The first call on a device looks up the array's device address with that
 * device current (cudaGetSymbolAddress).  Every call shares the one array and overwrites what an
 * earlier call left there (nothing of it is read back), so calls that may
 * overlap on the GPU (other streams, other host threads) race: order them
 * on one stream or serialise them. */
int hgks_flux_noalloc(const hgks_grid_t *grid, double gamma, double mu, double Pr, const int bc[6], const double *q,
                      double dt, double *L, double *dLdt, void *stream);

/* Kernel launches this handle has issued since creation (for accounting). */
unsigned long long hgks_launch_count(const hgks_t *h);

/* Measurement utility (the paper has no counterpart): the fused
 * multiply-add rate of the current device in one precision, in TFLOP/s
 * (2 flop per FMA), from independent FMA chains on every SM (one warm-up and
 * one timed launch of about 50 ms, CUDA events on cuda_stream; NULL is the
 * legacy default stream).  precision: HGKS_FP64 for the FP64 pipe,
 * HGKS_MIXED for the FP32 pipe.  It is the measured denominator of the ALU
 * roofline of the reconstruction and Gauss-point flux kernels.  Allocates
 * and frees a few KB of device memory; synchronises cuda_stream.
 * HGKS_E_INVALID for a bad precision or a NULL tflops. */
int hgks_alu_peak(int precision, void *cuda_stream, double *tflops);

/* Bytes of device memory this handle holds. */
unsigned long long hgks_device_bytes(const hgks_t *h);

/* One-line reason for the last failure on h (or on creation when h is NULL). */
const char *hgks_last_error(const hgks_t *h);

/* Free the handle and its device memory. */
void hgks_destroy(hgks_t *h);

#ifdef __cplusplus
}
#endif
#endif
