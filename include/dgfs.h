/*
 * dgfs.h - C ABI of the GB300 (sm_103a) fast Fourier spectral Boltzmann collision operator.
 *
 * The library evaluates the collision operator Q(f,g) of the Boltzmann equation
 * (arXiv:1809.10186, eq. eq_dim_Q_full, in the relative-velocity form eq. apndx_Q)
 * for the VHS kernel B = b |c - c_*|^gamma (eq. B_gen with alpha = 1), or the VSS kernel
 * B = b |c - c_*|^gamma (1 + cos chi)^(alpha - 1) (alpha in (1, 2]), with the fast
 * spectral method of the paper's Appendix (eqs. realGG, lowrank1, apndx_fs_Glm_Qk):
 * a batch of B independent distribution functions, each sampled on the uniform
 * cell-centred velocity grid c_j = -L + (j + 1/2) 2L/N of Sec. 3.3, goes in; Q at the
 * same grid points comes out. Each batch entry is one DG node of a physical mesh; the
 * 1/Kn factor of eq. eq_nbze is left to the caller.
 *
 * Memory layout of every field argument: [B][N][N][N], row-major, the third velocity
 * component fastest, contiguous. Element type: double for DGFS_PREC_FP64 plans, float
 * for every other precision. Field pointers are DEVICE pointers (except in
 * dgfs_collide_host), 16-byte aligned, owned by the caller. Outputs may not alias inputs.
 *
 * Streams: every compute call is stream-ordered and asynchronous on the given
 * cudaStream_t (passed as void*, NULL = legacy default stream). One plan owns one
 * workspace: calls with the same plan on different streams must be ordered by the caller.
 *
 * Errors: every call returns a dgfs_status. Argument errors return before any launch;
 * launch failures return DGFS_ERR_CUDA. A human-readable message for the last failure
 * of the calling thread is returned by dgfs_last_error_message(). No C++ exception
 * crosses this interface.
 *
 * Discretisation choices (the paper leaves them open):
 *  - M is the number of points of an antipodal FULL-sphere rule; the paper's
 *    half-sphere rule with M points is M_here = 2 M_paper.
 *  - Convolutions are circular on the grid (l + m wraps modulo N).
 *  - Nyquist modes (k = -N/2) are split evenly between -N/2 and +N/2, which makes every
 *    translate of a real grid function real (its multiplier is cos(pi N t / 2L)).
 *  - The loss weight G(m,m) is eq. lowrank1 at l = m (see dgfs_loss_mode).
 */
#ifndef DGFS_H
#define DGFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dgfs_plan_s* dgfs_plan_t;

typedef enum {
    DGFS_OK = 0,
    DGFS_ERR_INVALID_ARG = 1,  /* bad size, NULL or misaligned pointer, bad descriptor    */
    DGFS_ERR_UNSUPPORTED = 2,  /* valid request that the library does not implement       */
    DGFS_ERR_OOM = 3,          /* device or host allocation failed (plan creation only)    */
    DGFS_ERR_CUDA = 4,         /* a CUDA runtime call or kernel launch failed              */
    DGFS_ERR_TIMEOUT = 5,      /* a device-side bounded wait gave up (see stream_status)   */
    DGFS_ERR_NUMERIC = 6,      /* non-finite value detected in an output                   */
    DGFS_ERR_STATE = 7         /* destroyed or mismatched plan                              */
} dgfs_status;

typedef enum {
    DGFS_PREC_FP64 = 0,   /* CUDA-core FP64 everywhere (reference-accuracy mode; the VSS kernel
                             and dgfs_collide_noalloc up to N = 24)                                  */
    DGFS_PREC_FP32 = 1,   /* CUDA-core FP32 everywhere                                              */
    DGFS_PREC_F16S = 2,   /* translates on tcgen05 tensor cores: fp16 data operands with a per-node
                             power-of-two scale, every filter split into fp16 hi + lo parts (two
                             products), FP32 accumulation in tensor memory; FP32 elsewhere. N = 16, 32,
                             and 24 on the 32-point tiles (filters and data zero-padded: the exact
                             24-point result at (32/24)^3 the work of a 24-point tiling).
                             For every tensor-core precision, Q(f,f), Q(f,g), the JVP and dQ/dgamma
                             take their translates on the tensor cores (the bilinear calls by
                             polarisation: the translate-product sum is symmetric in f and g, so
                             P(f,g) = [P(f + a g) - P(f - a g)] / 4a with a = |f|/|g| per node); the
                             VJP runs on the FP32 CUDA-core translates. Accuracy (relative L2 of a
                             batch against the FP64 oracle on the N = 32 two-Maxwellian workload):
                             about 8e-4 of ||Q||, 5e-5 of the loss term ||Q-||                       */
    DGFS_PREC_BF16S = 3,  /* as F16S with bf16 operands (no scaling): about 7e-3 of ||Q||           */
    DGFS_PREC_F16X3 = 4,  /* translates on tcgen05 tensor cores with every data operand AND every
                             filter split into an fp16 hi part and a lo part times 2^11: three
                             products per contraction (hi hi, hi lo, lo hi), FP32 accumulation, so
                             the translates carry about FP32 accuracy (8e-6 of ||Q||, 4e-7 of ||Q-||,
                             as FP32); the two CTAs of a thread-block cluster share the field of one
                             (node, radial points) item. FP32 elsewhere. N = 16, 32, and 24 on the
                             32-point tiles as for F16S                                              */
    DGFS_PREC_BF16X3 = 5  /* as F16X3 with bf16 hi and lo parts (lo times 2^8), 16 significand
                             bits: about 2e-5 of ||Q||, within 1e-3 of ||Q|| at every node          */
} dgfs_precision;

typedef enum {
    /* G(m,m) = eq. lowrank1 at l = m: 4 pi sum_r w_r F(2m, c_r); the sphere sum is exact.
       This reading reproduces the paper's BKW error table (Sec. 4.3.1). */
    DGFS_LOSS_PAPER = 0,
    /* G(-m,m) of eq. lowrank1 from the gain's own sphere rule: Q^_0 = 0 exactly, so mass is
       conserved to round-off for any rule (less accurate loss for small rules). */
    DGFS_LOSS_CONSERVATIVE = 1
} dgfs_loss_mode;

typedef struct {
    int N;                     /* grid points per velocity axis: 8, 12, 16, 24 or 32 (tensor-core
                                  precisions: 16, 24 or 32; 24 on the 32-point tiles)         */
    double L;                  /* velocity domain [-L, L]^3 (Sec. 3.3), L > 0                   */
    double R;                  /* ball radius of the c_r integral; <= 0: 4L/(3+sqrt 2) (Appendix) */
    double gamma;              /* VHS exponent 2(1 - omega) of |c - c_*| (eq. B_gen)            */
    double b;                  /* kernel constant; <= 0: 1/(2^{3-omega} Gamma(5/2-omega) pi),
                                  omega = 1 - gamma/2 (Sec. 2.1, alpha = 1)                   */
    int M;                     /* full-sphere points; built-in rules for M = 6, 12, 26, 38      */
    const double* sphere_xyzw; /* optional host array [M/2][4]: one point (x,y,z) of each
                                  antipodal pair and the weight w of EACH of its two points,
                                  sum of w over the pairs = 2 pi; NULL: built-in rule for M   */
    int N_rho;                 /* Gauss-Legendre points on [0, R]; <= 0: N (Sec. 4.3.1)         */
    double svd_tol;            /* relative singular-value cut of the radial kernel; 0: none     */
    int svd_rank;              /* > 0: fixed rank of the radial kernel (overrides svd_tol)      */
    int precision;             /* dgfs_precision                                               */
    int loss_mode;             /* dgfs_loss_mode                                               */
    int64_t max_batch;         /* nodes processed per internal chunk (sizes the workspace:
                                  about 11 MB per node at N = 32, rank 19, plus up to 1.5 GB of
                                  transform batches); <= 0: chosen by the library
                                  (about 1.5 GB of workspace). Compute calls accept any B >= 0. */
    double alpha;              /* VSS scattering parameter of eq. B_gen, in [1, 2]; 0 or 1: VHS.
                                  alpha != 1 keeps the sphere point in the kernel factor
                                  F(k, c_r, sigma) of eq. realGG, so the gain takes one transform
                                  per radial AND sphere point (the paper's O(M N^4 log N) cost).
                                  Supported with DGFS_PREC_FP64 and DGFS_PREC_FP32, svd_tol = 0 and
                                  svd_rank = 0, by dgfs_collide, dgfs_collide2, dgfs_collide_jvp,
                                  dgfs_collide_host, dgfs_ssprk and the DG element calls; the
                                  others return DGFS_ERR_UNSUPPORTED. b <= 0 selects
                                  alpha / (2^{2-omega+alpha} Gamma(5/2-omega) pi) (Sec. 2.2).  */
} dgfs_plan_desc;

typedef struct {
    int N, N_rho, n_pairs, svd_rank_used, precision, loss_mode;
    double L, R, gamma, b;
    int64_t chunk_nodes;       /* nodes per internal chunk                                     */
    size_t workspace_bytes;    /* device workspace owned by the plan                           */
    size_t table_bytes;        /* device tables owned by the plan                              */
    double alpha;              /* VSS scattering parameter (1: VHS)                            */
} dgfs_plan_info_t;

/* Fill a descriptor with defaults (N=32, L=7, gamma=0, b=default, M=38, N_rho=N, FP32). */
dgfs_status dgfs_plan_desc_init(dgfs_plan_desc* desc);

/* Build the FP64 plan on the host (Gauss-Legendre rule, sphere rule, translate filters,
   radial kernel and its SVD, loss weights; Appendix eqs. realGG-lowrank1), round the
   tables to the device precision, allocate the device tables and workspace on the
   current device and copy the tables there (synchronously). The plan is owned by the
   caller until dgfs_plan_destroy. */
dgfs_status dgfs_plan_create(const dgfs_plan_desc* desc, dgfs_plan_t* plan_out);

/* Free the plan's device memory. Waits for the device first. NULL is accepted. */
dgfs_status dgfs_plan_destroy(dgfs_plan_t plan);

dgfs_status dgfs_plan_info(dgfs_plan_t plan, dgfs_plan_info_t* info);

/* Q(f,f) for B nodes (eq. apndx_fs_Glm_Qk for the gain, the G(m,m) convolution for the
   loss). f, Q: device [B][N^3]. */
dgfs_status dgfs_collide(dgfs_plan_t plan, const void* f, void* Q, int64_t B, void* stream);

/* Bilinear Q(f,g) of eq. anpdx_Q1: gain from f(c') g(c'_*), loss f(c) g(c_*). */
dgfs_status dgfs_collide2(dgfs_plan_t plan, const void* f, const void* g, void* Q,
                          int64_t B, void* stream);

/* Directional derivative dQ = Q(f,v) + Q(v,f) of Q(f,f) along v (Q is bilinear). */
dgfs_status dgfs_collide_jvp(dgfs_plan_t plan, const void* f, const void* v, void* dQ,
                             int64_t B, void* stream);

/* Transposed Jacobian: gf = (dQ(f,f)/df)^T u. Uses that every translate T_s of the
   symmetric-Nyquist discretisation satisfies T_s^T = T_{-s} and that the radial and loss
   multipliers are real and even: gf = sum_r sum_pairs 2 w_p [T_{-s}((K_r u) T_{-s} f)
   + T_s((K_r u) T_s f)] - u (K_L f) - K_L(u f). */
dgfs_status dgfs_collide_vjp(dgfs_plan_t plan, const void* f, const void* u, void* gf,
                             int64_t B, void* stream);

/* dQ(f,f)/dgamma at fixed b: the radial factor rho_r = 4 pi b c_r^{gamma+2} is replaced
   by its derivative ln(c_r) rho_r in both gain and loss. */
dgfs_status dgfs_collide_dgamma(dgfs_plan_t plan, const void* f, void* dQdg, int64_t B,
                                void* stream);

/* Q(f,f) for nodes of mixed grid size (one plan per N) and per-node kernel parameters.
   plans[nplans]: plans of equal precision. Host arrays of length B: node_plan[i] (index
   into plans), node_offset[i] (element offset of node i in the packed f and Q; each node
   occupies N_i^3 elements), node_gamma[i] and node_b[i] (NULL: the plan's values).
   f, Q: device, packed. */
dgfs_status dgfs_collide_ragged(const dgfs_plan_t* plans, int nplans, const int32_t* node_plan,
                                const int64_t* node_offset, const double* node_gamma,
                                const double* node_b, int64_t B, const void* f, void* Q,
                                void* stream);

/* A ragged schedule: the node layout of dgfs_collide_ragged (plan per node, offsets, per-node
   gamma and b) prepared once, for a mesh whose layout does not change between calls (a DG mesh
   over time steps). dgfs_ragged_create validates the layout exactly as dgfs_collide_ragged does,
   groups the nodes by plan and copies the per-class offsets, gamma and b to device memory the
   schedule owns (it allocates; the call is synchronous). dgfs_ragged_collide then computes
   Q(f,f) for every node with stream-ordered kernel launches only, no host staging, so a whole
   mixed-N batch can be captured in one CUDA graph. When the classes with nodes use distinct plans,
   they run concurrently on streams the schedule owns, forked from `stream` at the call and joined
   back to it before the call's later work (a graph capture records them as parallel branches). The
   plans must outlive the schedule; calls through one schedule (or its plans) must not run
   concurrently on different streams.
   The paper has no counterpart (its element-local parallelism, Sec. 3, is the reason nodes are
   independent). Arguments as dgfs_collide_ragged; node_plan, node_offset, node_gamma, node_b
   are HOST arrays, read during the create call only. */
typedef struct dgfs_ragged_s* dgfs_ragged_t;
dgfs_status dgfs_ragged_create(const dgfs_plan_t* plans, int nplans, const int32_t* node_plan,
                               const int64_t* node_offset, const double* node_gamma,
                               const double* node_b, int64_t B, dgfs_ragged_t* out);
dgfs_status dgfs_ragged_collide(dgfs_ragged_t ragged, const void* f, void* Q, void* stream);
/* Releases the schedule's device arrays and streams (synchronises the device first). NULL is a no-op. */
dgfs_status dgfs_ragged_destroy(dgfs_ragged_t ragged);

/* ---- 1-D DGFS solver (Sec. 3: eq. eq_weakForm, the upwind flux eq. eq_numericalFlux_upwind,
   the fully diffuse wall condition of Sec. 3.6, eqs. SSPRK2/SSPRK3) ------------------------------
   A slab x in [edges[0], edges[I]] of I elements, K Gauss-Lobatto nodes each (nodal DG basis), walls
   at both ends. F: device [I][K][N^3] (element-major, the plan's element type), node l of element i
   at x = (edges[i] + edges[i+1])/2 + (edges[i+1] - edges[i])/2 * xi_l. The right-hand side is
     dF/dt = (2/h_i) M^{-1} (c_1 S F - Fl) + (1/Kn) M^{-1} sum_{l1,l2} H Q(F_l1, F_l2)
   with S[m][l] = int phi_l phi_m' and M, H on [-1, 1], the upwind flux Fl (interior value where
   c_1 n >= 0, neighbour or wall value otherwise) and, at a wall with velocity u_w (u_w,x = 0) and
   temperature T_w, the incoming value n_w exp(-|c - u_w|^2 / T_w), n_w balancing the outgoing
   mass flux of the wall node. The collision term is the DG element term of dgfs_dg_collide (the
   SVD variant at svd_tol) with the plan's kernel (VHS or VSS). Kn = +infinity: collisionless.
   wall_left, wall_right: host arrays {u_x, u_y, u_z, T_w} in the units of the velocity grid.
   dgfs_slab_create and dgfs_slab_set_walls synchronise the device; the other calls are
   stream-ordered. A slab must not be used concurrently on several streams, nor its plan. */
typedef struct dgfs_slab_s* dgfs_slab_t;
dgfs_status dgfs_slab_create(dgfs_plan_t plan, int K, int I, const double* edges, double Kn,
                             const double* wall_left, const double* wall_right, double svd_tol,
                             dgfs_slab_t* out);
dgfs_status dgfs_slab_set_walls(dgfs_slab_t slab, const double* wall_left, const double* wall_right);
/* dFdt = the right-hand side at F (both device [I][K][N^3], distinct). */
dgfs_status dgfs_slab_rhs(dgfs_slab_t slab, const void* F, void* dFdt, void* stream);
/* nsteps SSP-RK steps (order 2 or 3) of size dt, in place on F. With nsteps >= 2, a plan that is not
   profiling and a stream that is not being captured, the first step runs eagerly and one step is then
   captured as a CUDA graph (on a slab-owned stream) and replayed for the rest; the graph is kept for
   later calls with the same F, dt, order and plan tuning, and dropped by dgfs_slab_set_walls.
   Otherwise every step is launched eagerly (on a capturing stream, into the caller's graph), and so
   are the remaining steps when capturing or instantiating the graph fails (that error is cleared).
   Both give the same bits. The graph is keyed by F's address: a new field buffer at the same address
   (of the slab's fixed size) reuses it. */
dgfs_status dgfs_slab_ssprk(dgfs_slab_t slab, int order, void* F, double dt, int nsteps, void* stream);
dgfs_status dgfs_slab_destroy(dgfs_slab_t slab);
/* Host: S [K][K] (eq. eq_stiffMatrix1 on [-1, 1]) and the inverse mass matrix [K][K]; either NULL. */
dgfs_status dgfs_host_dg_stiffness(int K, double* S, double* Minv);

/* dgfs_collide with HOST buffers: copies f to the device, computes, copies Q back and
   synchronises before returning. f_host/Q_host may be pageable or pinned (pinned lets the
   copies overlap the compute). The batch is split into sub-batches that fit the plan's staging
   buffers (at most half the plan's chunk each): their sizes ramp up from B / 32 nodes by a factor
   of 4 and down again at the end (only the first input copy and the last output copy are not
   hidden), with as few as fit in between. The copies run on two copy streams owned by the plan,
   so the host-to-device copy of one sub-batch and the device-to-host copy of the previous one
   overlap the compute on `stream`. */
dgfs_status dgfs_collide_host(dgfs_plan_t plan, const void* f_host, void* Q_host, int64_t B,
                              void* stream);

/* Q(f,f) as dgfs_collide computes it (the same kernels, except that FP32/FP64 plans form the
   translate products with the dense circulant kernel where dgfs_collide takes them in Fourier
   space: equal to rounding), for callers that must not allocate device
   memory when they run (for example code whose device memory is fully reserved up front, or
   that may not pay the device synchronisation an allocation can cause). The paper has no
   counterpart to this call. Its intermediate fields live in one fixed 64 MiB device array
   defined in this library (one per GPU that loads it, held until the process exits) instead of
   the plan's workspace; it calls no allocating routine. B is limited to the number of nodes
   whose scratch fits the array: floor(64 MiB / s) with s = e (N_rho + 2 (rank + 2) + 4) N^3
   bytes per node (e = 4 for float plans, 8 for FP64; each of the three parts rounded up to
   256 bytes), i.e. 6 nodes at N = 32, N_rho = 32 with an SVD rank of 19, 4 at N = 32 without
   truncation, 73 at N = 16, N_rho = 16; larger B returns DGFS_ERR_INVALID_ARG with the limit
   in the message. The first call on a device looks up the
   array's device address; make it before capturing any stream. Every call shares the array:
   calls whose work overlaps on the GPU race on it. f, Q: device, [B][N^3], as dgfs_collide. */
dgfs_status dgfs_collide_noalloc(dgfs_plan_t plan, const void* f, void* Q, int64_t B, void* stream);

/* Synchronise the stream and report device-side flags raised by earlier calls with this
   plan (DGFS_ERR_TIMEOUT, DGFS_ERR_NUMERIC), then clear them. */
dgfs_status dgfs_stream_status(dgfs_plan_t plan, void* stream);

/* ---- space-homogeneous time stepping and moments (Secs. 3.3, 3.5) ---------------------
   dgfs_ssprk advances df/dt = scale Q(f, f) (scale: e.g. 1/Kn) by nsteps steps of dt with the
   2nd- or 3rd-order SSP Runge-Kutta scheme (eqs. SSPRK2, SSPRK3), in place: f device [B][N^3] in
   the plan's element type. Every stage is a dgfs_collide evaluation plus one elementwise
   combination kernel; the stage fields live in the plan's workspace. Stream-ordered, no
   allocation; non-finite values raise DGFS_ERR_NUMERIC in dgfs_stream_status. */
dgfs_status dgfs_ssprk(dgfs_plan_t plan, int order, void* f, int64_t B, double dt, double scale, int nsteps,
                       void* stream);
/* Mid-point-rule moments of every node (eq. moments1) and Boltzmann's H: out device [B][15]
   doubles: n, u_x, u_y, u_z, T, P_xx, P_yy, P_zz, P_xy, P_xz, P_yz, q_x, q_y, q_z, H, with
   T = 2/(3n) int f |c-u|^2, P = 2 int f (c-u)(c-u), q = int f (c-u)|c-u|^2, H = int f ln f over
   the points where f > 0; accumulated in FP64. */
dgfs_status dgfs_moments(dgfs_plan_t plan, const void* f, double* out, int64_t B, void* stream);

/* ---- DG element collision term (Sec. 3.4) ---------------------------------------------
   In the weak form (eq. eq_weakForm) the collision term of test function m in an element is
     C[m] = sum_{l1, l2} H[m][l1][l2] Q(F[l1], F[l2])                               (eq. HH)
   with H[m][l1][l2] = int phi_m phi_l1 phi_l2 (eq. eq_stiffMatrix3) and F[l] the element's K
   nodal distribution functions. dgfs_dg evaluates it in the paper's SVD variant (eqs.
   eq_coln_derivation_SVD_3/4): each K x K slice H[m] = sum_r U[l1][r] V[r][l2] (singular values
   in V), C[m] = sum_r Q(f_r, g_r), f_r = sum_l U[l][r] F[l], g_r = sum_l V[r][l] F[l]: R_m <= K
   bilinear collisions per m instead of K^2. The 1/Kn factor is left to the caller. */
typedef struct dgfs_dg_s* dgfs_dg_t;
/* H: host [K][K][K] (read during the call), 2 <= K <= 16. svd_tol: singular values of H[m] at
   or below svd_tol times its largest are dropped (0: keep those above 1e-14 of the largest).
   max_elements: elements per internal pass (sizes the device workspace: 3 R max_elements N^3
   values, R = sum_m R_m); calls accept any E. The plan must outlive the object. */
dgfs_status dgfs_dg_create(dgfs_plan_t plan, int K, const double* H, double svd_tol, int64_t max_elements,
                           dgfs_dg_t* out);
/* ranks: host [K] or NULL (R_m of every m); total: host or NULL (R). */
dgfs_status dgfs_dg_info(dgfs_dg_t dg, int* ranks, int* total);
/* F, C: device [E][K][N^3] in the plan's element type (float; double for FP64 plans), 16-byte
   aligned, not aliased; C[e][m] as above. Stream-ordered; no allocation. The collisions run as
   dgfs_collide / dgfs_collide2 compute them in the plan's precision (on the tensor cores for the
   tensor-core precisions). */
dgfs_status dgfs_dg_collide(dgfs_dg_t dg, const void* F, void* C, int64_t E, void* stream);
/* Synchronises the device and frees the workspace. NULL is a no-op. */
dgfs_status dgfs_dg_destroy(dgfs_dg_t dg);
/* Host only: the 1-D nodal basis of the paper's slab cases: the K Gauss-Lobatto points of the
   reference element [-1, 1] (nodes[K]), its mass matrix M[m][l] (eq. eq_massMatrix, [K][K]) and
   H[m][l1][l2] ([K][K][K]), by Gauss-Legendre quadrature exact for the polynomial integrands. */
dgfs_status dgfs_host_dg_tensor(int K, double* nodes, double* M, double* H);

/* Test hook of the failure detection (the paper has no counterpart). mode 1: in the next
   compute call of a tensor-core plan, the first CTA of the translate-product kernel withholds
   the signal that its pass-3 operands are complete, as a lost hand-off would. Its bounded
   waits then give up, every role of that CTA stops, the MMAs in flight are drained, TMEM is
   freed, its P_r is not written and flag TIMEOUT is raised; the other CTAs and later calls are
   unaffected. mode 0 clears the injection. Other plans and precisions ignore it. */
dgfs_status dgfs_debug_inject(dgfs_plan_t plan, int mode);

/* Profiling of one plan: between begin and end the library counts its kernel launches and
   brackets every launch of the translate-product kernel (the dominant kernel) with CUDA
   events on the call's stream. end synchronises those events and reports the totals.
   At most 65536 bracketed launches per session; later ones are counted, not timed. */
typedef struct {
    int64_t launches;         /* kernels launched by compute calls of this plan             */
    int64_t gain_launches;    /* translate-product kernel launches                           */
    int64_t gain_timed;       /* of which bracketed by events                                */
    double gain_ms;           /* summed event time of the bracketed launches                 */
    int64_t nodes;            /* node evaluations requested                                  */
} dgfs_profile_t;

dgfs_status dgfs_profile_begin(dgfs_plan_t plan);
dgfs_status dgfs_profile_end(dgfs_plan_t plan, dgfs_profile_t* out);

/* Autotuner (the paper has no counterpart): times dgfs_collide on the caller's batch f (device,
   [B][N^3], the plan's element type; the first min(B, chunk) nodes are used) for every candidate
   configuration - radial points per work item of the persistent tensor-core translate kernel (per
   CTA pair of the split-data kernels; 1, 2, 4, 8 where
   they divide N_rho, or the batch-size rule) times nodes per internal chunk (the plan's chunk and
   its halves) - with CUDA events on `stream`, keeps the fastest in the plan for its later compute
   calls and caches it in the process by (N, sphere pairs, N_rho, SVD rank, precision, batch size
   rounded down to a power of two): a later call for the same shape applies the cached choice
   without timing (report->cached = 1). Results do not depend on the choice (each radial point's
   arithmetic is the same in every configuration). Synchronous; not for use inside a stream
   capture. The output goes to the plan's own staging buffer. VSS plans: DGFS_ERR_UNSUPPORTED. */
typedef struct {
    int rpc;                        /* radial points per item chosen (0 for plans without tensor cores) */
    int64_t chunk_nodes;            /* nodes per chunk chosen                                          */
    double ms_per_node_default;     /* time per node with the batch-size rule and the plan's chunk     */
    double ms_per_node_tuned;       /* time per node with the choice                                   */
    int candidates;                 /* configurations timed (0 when the choice came from the cache)    */
    int cached;
} dgfs_tune_report;
dgfs_status dgfs_plan_autotune(dgfs_plan_t plan, const void* f, int64_t B, void* stream, dgfs_tune_report* report);
/* Sets the configuration by hand: rpc dividing N_rho (0: the batch-size rule), chunk_nodes >= 0
   (0: the plan's chunk). */
dgfs_status dgfs_plan_set_tuning(dgfs_plan_t plan, int rpc, int64_t chunk_nodes);

/* Device-rate probe for rooflines (the paper has no counterpart): the FP32 and FP64 fused
   multiply-add throughput of the CUDA cores of the current device, in TFLOP/s (2 flops per FMA),
   the best of three timed launches of independent FMA chains on every SM. Synchronous; allocates
   a few bytes of device memory for the duration of the call; changes no device setting. Either
   output may be NULL. */
dgfs_status dgfs_device_fma_peaks(double* fp32_tflops, double* fp64_tflops);

/* Tensor-core rate probe (the paper has no counterpart): SM clock cycles per tcgen05.mma.kind::f16
   of the shape M = 128, K = 16, N = n (a multiple of 16 in [16, 256]) issued back to back into one
   FP32 accumulator, on the slowest SM of the current device (one CTA per SM, 4096 MMAs, the second
   of two launches). The A operand comes from shared memory (a_from_tmem = 0; MN-major, no swizzle,
   as the translate kernels' pass-2/3 operands) or from tensor memory (1; as their pass-1 operand).
   Sets the ceiling that the MMA shapes of a kernel allow: 2 * 128 * n * 16 flops per MMA over these
   cycles. Synchronous; allocates a few bytes of device memory; changes no device setting. */
dgfs_status dgfs_device_mma_cycles(int n, int a_from_tmem, double* cycles_per_mma);

/* The fingerprint of a plan (dgfs_host_plan_fingerprint of its descriptor). */
dgfs_status dgfs_plan_fingerprint(dgfs_plan_t plan, uint64_t* fingerprint);

/* Message of the last failed call on the calling thread ("" if none). */
const char* dgfs_last_error_message(void);

/* ---- host-only introspection of the plan builder (no CUDA call, usable without a GPU) */

/* Quadrature of a descriptor: c_r[N_rho], w_r[N_rho] (Gauss-Legendre on [0,R]),
   sigma_xyzw[n_pairs][4] (pair representatives and per-point weights). *n_pairs receives
   M/2; arrays may be NULL to query sizes only. */
dgfs_status dgfs_host_quadrature(const dgfs_plan_desc* desc, double* c_r, double* w_r,
                                 double* sigma_xyzw, int* n_pairs, double* R_used,
                                 double* b_used);

/* Fingerprint of the plan a descriptor builds: a 64-bit FNV-1a hash of its precision, sizes,
   scalars and every FP64 table of the host plan (quadrature, sphere rule, translate filters,
   radial-kernel factors, loss weights, VSS factors), in a fixed order. Equal fingerprints mean the
   same arithmetic; the tables come from the host's libm, so machines of different architecture can
   give different fingerprints for one descriptor. No GPU needed. */
dgfs_status dgfs_host_plan_fingerprint(const dgfs_plan_desc* desc, uint64_t* fingerprint);

/* Sub-batch sizes dgfs_collide_host uses for B nodes on a plan whose chunk is `chunk` nodes: at most
   chunk / 2 each (chunk >= 2; 1 for a one-node chunk), ramping up from B / 32 by a factor of 4 and
   down again, with as few as fit in between; they sum to B. Writes min(count, cap) sizes (sizes may
   be NULL to query the count) and the count to *count. B >= 0, chunk >= 1, else DGFS_ERR_INVALID_ARG.
   No GPU needed. */
dgfs_status dgfs_host_pipeline_schedule(int64_t B, int64_t chunk, int64_t* sizes, int64_t cap, int64_t* count);

/* Circulant translate filter a[N] of the shift t along one axis: (T_t f)_j =
   sum_j' a[(j - j') mod N] f_j', the grid restriction of the trigonometric interpolant
   shifted by t (multiplier e^{i pi k t / L}, Nyquist: cos(pi N t / 2L)). */
dgfs_status dgfs_host_translate_filter(int N, double L, double t, double* a);

/* The plan builder's VSS kernel factor F(k, c_r, sigma) of eq. realGG for B = b c_r^gamma
   (1 + cos chi)^(alpha - 1) (Funk-Hecke series of its Legendre expansion), at n points given
   by k_abs[i] = |k| (lattice units), mu[i] = sigma.k / |k| and c_r[i]; host arrays, F[i] out.
   b <= 0 selects the default constant of dgfs_plan_desc. No GPU needed. */
dgfs_status dgfs_host_vss_factor(double L, double gamma, double b, double alpha, int n,
                                 const double* k_abs, const double* mu, const double* c_r, double* F);

/* The FP64 tables a VSS plan (desc->alpha != 1) would upload, built on the host: A [N_rho][n_pairs]
   [N^3] = w_r w_p F(k, c_r, sigma_p) and the loss weight GL [N^3], both in DFT index order (index
   q of an axis is the lattice index q for q < N/2, q - N otherwise). Host arrays sized by the caller
   (n_pairs as returned by dgfs_host_quadrature); either may be NULL. No GPU needed. */
dgfs_status dgfs_host_vss_tables(const dgfs_plan_desc* desc, double* A, double* GL);

#ifdef __cplusplus
}
#endif

#endif /* DGFS_H */
