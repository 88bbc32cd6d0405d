/*
 * xlbomd.h - C ABI of the GB300 XL-BOMD hot path.
 *
 * Finite-temperature extended-Lagrangian Born-Oppenheimer molecular dynamics
 * (A. M. N. Niklasson, arXiv:1705.10845) on an orthogonal self-consistent-
 * charge tight-binding (SCC-TB) model.  One MD step (Section II.E, Eqs.
 * Integration and VRL_Damp) builds H[n] from the dynamical charges n, forms
 * the density matrix D = f(H[n]) by the recursive Fermi-operator expansion
 * with the chemical potential fixed by Tr D = N_occ (Section IV.B), computes
 * the charge response along m probe directions by canonical density-matrix
 * perturbation theory (Section V.B), applies the rank-m kernel
 * K ~ (dq/dn - I)^-1 (Section V.D-V.E, Eqs. KCI, JCI, K_up, v_1), takes the
 * Mulliken charges and Hellmann-Feynman forces (Eq. EqMotFT) and advances R
 * and n (Eq. VRL_Damp with Table I).
 *
 * Conventions (every entry point):
 *  - All device state is owned by the context; the library allocates it in
 *    xlbomd_init and frees it in xlbomd_free.  Host arrays passed in are
 *    copied before the call returns; the caller keeps ownership.
 *  - Work is enqueued on the CUDA stream given to xlbomd_init (NULL = the
 *    legacy default stream).  Calls that must read device results to decide
 *    the next launch (the chemical-potential Newton loop, the probe loop of
 *    the kernel update, xlbomd_get) synchronise that stream.
 *  - Errors never abort the process and no kernel traps.  A failing call
 *    returns a negative status; the status is also stored in the context
 *    (sticky: later calls return it without doing work until
 *    xlbomd_clear_error) and xlbomd_last_error() gives a message.
 *  - Units: Angstrom, eV, fs, amu, Kelvin; charges in electrons.
 *  - Layouts: positions, velocities, forces are natoms x 3 row-major double;
 *    charge vectors are natoms doubles; matrices are N x N row-major double
 *    with N = 4 natoms (orbital order s, px, py, pz per atom).
 */
#ifndef XLBOMD_API_H_
#define XLBOMD_API_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef struct xlbomd_ctx xlbomd_ctx;

typedef enum {
  XLBOMD_OK = 0,
  XLBOMD_ERR_ARG = -1,           /* invalid argument or size */
  XLBOMD_ERR_OOM = -2,           /* device allocation failed */
  XLBOMD_ERR_CUDA = -3,          /* a CUDA call failed */
  XLBOMD_ERR_NOT_CONVERGED = -4, /* SCF or chemical-potential iteration budget spent */
  XLBOMD_ERR_SPECTRUM = -5,      /* |beta (e - mu)| / 2^(n+1) >= 1 for a Gershgorin bound */
  XLBOMD_ERR_DIVERGED = -6,      /* residual |q - n| above the divergence threshold */
  XLBOMD_ERR_TIMEOUT = -7,       /* a bounded device wait gave up, or a product tile fell outside the matrix */
  XLBOMD_ERR_UNSUPPORTED = -8    /* requested precision not built for this device */
} xlbomd_status;

/* Arithmetic of the expansion and response matrix products. */
typedef enum {
  XLBOMD_FP64 = 0,   /* plain FP64 products */
  XLBOMD_FP16x3 = 1, /* split FP16 hi/lo operands, 3 products, FP32 accumulation */
  XLBOMD_BF16x3 = 2, /* split BF16 hi/lo operands, 3 products, FP32 accumulation */
  XLBOMD_TF32x3 = 3  /* split TF32 hi/lo operands (FP32 words), 3 products of tcgen05 kind::tf32,
                        FP32 accumulation; twice the operand bytes and half the tensor rate of
                        the 16-bit forms */
} xlbomd_prec;

/* Model and integrator constants.  xlbomd_default_params() fills the values
 * of the 24-atom reference system (Te = 1000 K, 10 squarings, rank 2). */
typedef struct {
  /* Slater-Koster model (Section VI stand-in) */
  double eps_s, eps_p;     /* on-site energies (eV) */
  double t0[4];            /* ss-sigma, sp-sigma, pp-sigma, pp-pi prefactors (eV) */
  double r_decay;          /* hopping decay length (A) */
  double r_cut, r_taper;   /* quintic taper on [r_taper, r_cut] (A) */
  double hubbard_U;        /* on-site Coulomb (eV) */
  double coulomb_k;        /* e^2 / (4 pi eps0) = 14.399645 eV A */
  /* electrons */
  double Te;               /* electronic temperature (K) */
  int n_sq;                /* squarings of the recursive Fermi-operator expansion */
  /* XL-BOMD (Table I row kmax) */
  double dt;               /* fs */
  double kappa, alpha;
  double c[8];
  int kmax;                /* 5, 6 or 7 */
  int rank_m;              /* probes per kernel update, 0..8 */
  double kernel_c;         /* J_0 = c I, c != 1 (Eq. JCI) */
  double mix_alpha;        /* linear mixing of the t0 SCF */
  double scf_tol;          /* max |q - n| of the t0 SCF */
  int scf_max_iter;
  double mu_tol;           /* |beta dmu| below which the Newton loop on mu stops */
  int mu_max_iter;
  double diverge_tol;      /* max |q - n| above which a step reports ERR_DIVERGED */
  int prec;                /* xlbomd_prec */
  int energy_every;        /* energy monitor every k steps inside xlbomd_step (0 = never) */
  int scf_mode;            /* t0 SCF: 0 = linear mixing, 1 = n <- n - K_m (q - n) with the rank-m
                              kernel (Eq. SCF_K), for systems whose charge sloshing is too stiff
                              for linear mixing */
  int kernel_auto;         /* 1: at the start of xlbomd_scf, set c of J_0 = c I per system to
                              1.2 x the most negative eigenvalue of dq/dn (power iteration on
                              the response, 12 probes), so that K_0 = (c - 1)^-1 I keeps the
                              stiffest charge mode stable */
  int kernel_mode;         /* 0: rank-m kernel rebuilt every step (Eq. K_up, v_1);
                              1: exact kernel K = (J - I)^-1 of Eq. KK, J = dq/dn from the
                              responses to the natoms unit directions, held between
                              recomputations (Section VI.A);
                              2: accumulated kernel: K and J carried from step to step, one
                              rank-1 update per kernel update with v = K r/|K r|; a started
                              kernel (first update, or xlbomd_scf) is K_0 = (c - 1)^-1 I,
                              J_0 = c I without an update (end of Section V.F) */
  int kernel_every;        /* kernel_mode 1: recompute K every this many MD steps
                              (0: keep the kernel of the t0 state) */
  double rep_A;            /* optional pair repulsion rep_A exp(-r/rep_rho) S(r) over the image
                              pairs within r_cut, S the hoppings' taper (eV; 0 = off, the
                              default).  The model has no repulsive term otherwise, and its
                              atoms fall into each other within a few hundred steps */
  double rep_rho;          /* its decay length (A) */
  int kernel_prec;         /* split precisions: 0 = the kernel's response chains (probes, the
                              stiffest-mode search, exact-kernel columns) take the three products
                              of the split; 1 = one product of the hi operands (FP32
                              accumulation).  The kernel only preconditions the n dynamics and
                              the forces do not contain it; the expansion always takes three,
                              the chemical-potential chain follows mu_prec.  Ignored by FP64. */
  int graphs;              /* 1: split precisions with at most 2048 padded orbitals capture each
                              chemical-potential pass (per Newton-Schulz plan) and each probe's
                              response in CUDA graphs and replay them (the second run of a plan
                              is captured; results are bitwise those of direct launches).  Needs
                              a caller stream (xlbomd_init's cuda_stream, not the legacy default
                              stream, which cannot be captured).  On many concurrent 32-512-atom
                              trajectories it measured slower than direct launches, so it is
                              off by default.  0: off. */
  int mu_prec;             /* split precisions: 0 = the chemical-potential chain (dD/dmu) takes the
                              three products of the split; 1 = one hi*hi product.  dD/dmu only
                              sets the Newton step on mu and the first-order correction
                              D(mu + dmu) = D(mu) + dmu dD/dmu, whose trace stays exact whatever
                              its error; D's error from it is at most |dmu| times the error of
                              dD/dmu, and the last Newton step has |dmu| < mu_tol / beta.
                              Ignored by FP64. */
} xlbomd_params;

/* One trajectory.  R and V are natoms x 3 row-major (A, A/fs), Z natoms
 * valence charges (4 for the carbon-like model), mass in amu. */
typedef struct {
  int natoms;
  double box_L;
  const double* R;
  const double* V;
  const double* Z;
  double mass;
} xlbomd_system;

/* Quantities for xlbomd_get / xlbomd_set. */
typedef enum {
  XLBOMD_Q = 0,        /* get: Mulliken charges q[n] (natoms) */
  XLBOMD_N = 1,        /* get/set: n(t) (natoms); set fills the whole history with it */
  XLBOMD_NHIST = 2,    /* get/set: n(t - k dt), k = 0..kmax ((kmax+1) x natoms) */
  XLBOMD_F = 3,        /* get: forces (natoms x 3, eV/A) */
  XLBOMD_R = 4,        /* get/set: positions (natoms x 3) */
  XLBOMD_V = 5,        /* get/set: velocities (natoms x 3) */
  XLBOMD_KR = 6,       /* get: K (q - n) (natoms) */
  XLBOMD_RES = 7,      /* get: residual q - n (natoms) */
  XLBOMD_ENERGY = 8,   /* get: [Omega, band, coulomb, entropy, kinetic, total, repulsion] (7);
                          Omega includes the repulsion */
  XLBOMD_MU = 9,       /* get/set: chemical potential (1); set is the Newton start */
  XLBOMD_D = 10,       /* get: density matrix (N x N) */
  XLBOMD_H = 11,       /* get: H[n] (N x N) */
  XLBOMD_GAMMA = 12,   /* get: Coulomb matrix gamma (natoms x natoms) */
  XLBOMD_STATS = 13,   /* get: [mu passes, NS products, probes used, GEMMs, steps] (5) */
  XLBOMD_PROBES = 14,  /* get: probes V then responses W (2 x rank_m x natoms) */
  XLBOMD_KMAT = 15     /* get: held kernel K (natoms x natoms, row-major; kernel_mode 1, 2) */
} xlbomd_quantity;

/* Defaults of the 24-atom reference workload. */
void xlbomd_default_params(xlbomd_params* p);

/* Table I row kmax (5, 6 or 7): kappa, alpha and c_0..c_kmax of the dissipative
 * n update (Eq. VRL_Damp) written into p (kmax, kappa, alpha, c; the other
 * fields are untouched).  Errors: ERR_ARG for another kmax or a null p. */
xlbomd_status xlbomd_table_i(xlbomd_params* p, int kmax);

/* Allocate device state for nsys trajectories and upload R, V, Z (Eq. IBC
 * nuclear initial conditions).  Builds H0 and gamma; n = 0.  Does not run
 * the t0 SCF (xlbomd_scf).  cuda_stream is a cudaStream_t or NULL.
 * Errors: ERR_ARG (natoms < 1, box_L <= r_cut, rank_m > 8, kmax not 5..7,
 * n_sq < 1, kernel_c == 1, nsys < 1), ERR_OOM, ERR_CUDA, ERR_UNSUPPORTED. */
xlbomd_status xlbomd_init(const xlbomd_params* params, const xlbomd_system* systems, int nsys,
                          void* cuda_stream, xlbomd_ctx** out);

/* t0 ground state of system sys (Eq. IBC): SCF to max|q - n| < scf_tol by
 * linear mixing n <- n + mix_alpha (q[n] - n) (Eq. SCF_K with K_0, scf_mode 0)
 * or by n <- n - K_m (q[n] - n) with the rank-m kernel (Eq. SCF_K, scf_mode 1);
 * then n-history = n(t0), forces and K r at t0.  sys = -1: every system, those
 * of one padded orbital count in lockstep (grouped densities, stiffest-mode
 * search and kernel updates; each system takes its one-system iterations).
 * Split precisions also stop at the rounding floor of their products: when
 * max|q - n| is below 100 scf_tol and has not fallen by 10% in 4 iterations.
 * Errors: ERR_NOT_CONVERGED (scf_max_iter spent), ERR_DIVERGED (non-finite or
 * max|q - n| > 1e3), and those of xlbomd_density. */
xlbomd_status xlbomd_scf(xlbomd_ctx* ctx, int sys);

/* H0, gamma and H[n] at the current R (rows a1-a2 of the path).  H[n] is the
 * Hamiltonian of the linearised functional at the dynamical charges n
 * (Section IV.A, the Kohn-Sham shadow potential: H_KS[n] with the Hartree
 * term evaluated at n): in the SCC-TB model H[n] = H0 + diag(gamma n) per
 * orbital, gamma the Coulomb matrix (Hubbard U on the diagonal).  Enqueued
 * asynchronously; clears the context's density (a later xlbomd_density must
 * run before xlbomd_response / xlbomd_kernel_update).  Errors: ERR_ARG (bad
 * sys), ERR_CUDA. */
xlbomd_status xlbomd_build_H(xlbomd_ctx* ctx, int sys);

/* a3-a6: recursive expansion D = f(H[n]) with mu from Tr D = N_occ
 * (Section IV.B), Mulliken q, residual r = q - n, forces (Eq. EqMotFT). */
xlbomd_status xlbomd_density(xlbomd_ctx* ctx, int sys);

/* a7 for one probe: w = d q[n + lambda v] / d lambda (Section V.B, canonical
 * perturbation theory, mu re-solved to hold N_occ).  v_dev, w_dev are device
 * arrays of natoms doubles; requires xlbomd_density on the same state. */
xlbomd_status xlbomd_response(xlbomd_ctx* ctx, int sys, const double* v_dev, double* w_dev);

/* The same one-probe response as xlbomd_response, for callers that must not
 * allocate device memory while they run: code that holds a fixed memory
 * budget, runs next to a caching allocator it may not disturb, or replays
 * work where a cudaMalloc or cudaFree would stall every other stream.  This
 * call allocates nothing: the response chain's work matrices and vectors live
 * in one file-scope static device array of about 2.6 MB, which every GPU that
 * loads this library holds until the process exits.  The caller still passes
 * the probe v_dev and the output w_dev (device arrays of natoms doubles), and
 * the context must be an FP64 one (prec = XLBOMD_FP64) whose xlbomd_density
 * has run.  Limit: padded orbital count <= 256 (at most 64 atoms); larger
 * systems get XLBOMD_ERR_ARG with a message, other precisions
 * XLBOMD_ERR_UNSUPPORTED.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress), so make that first call before any
 * stream capture.  All calls share the one array and it keeps the last call's
 * contents: calls that overlap on the GPU (other streams, other contexts,
 * other host threads) race on it.  Every argument check (including the
 * reciprocal-vector count of the Coulomb sum) comes before the first
 * operation on the shared array, and its products are counted in
 * XLBOMD_STATS like those of xlbomd_response.  The paper has no counterpart to
 * this entry point; it exists for callers that cannot allocate. */
xlbomd_status xlbomd_response_noalloc(xlbomd_ctx* ctx, int sys, const double* v_dev, double* w_dev);

/* a7-a8: K r into KR.  kernel_mode 0: rank-m kernel on r (Eqs. K_up, v_1;
 * Woodbury form).  kernel_mode 1: the held exact kernel applied to r (computed
 * first, by xlbomd_kernel_exact, when none is held).  kernel_mode 2: one rank-1
 * update of the carried kernel at the current state, then K r (the first call,
 * and the call that ends xlbomd_scf, start the kernel at K_0 instead). */
xlbomd_status xlbomd_kernel_update(xlbomd_ctx* ctx, int sys);

/* Exact kernel K = (J - I)^-1 (Eq. KK) at the current density: J = dq/dn
 * column by column from the responses to the natoms unit directions (the
 * full-rank end of the Eq. K_up sequence), inverted on the device in FP64 by
 * Gauss-Jordan elimination with partial pivoting.  Costs natoms responses.
 * The kernel is held in the context (XLBOMD_KMAT) and used by
 * xlbomd_kernel_update, xlbomd_scf and xlbomd_step when kernel_mode = 1.
 * Split precisions run the unit-probe response chains up to 64 at a time, each
 * in a chain slot of its own (response-chain matrices, allocated on the first
 * call within a quarter of the free device memory and kept by the context),
 * every chain product one grouped launch over the probes.
 * Requires xlbomd_density on the same state.  Errors: ERR_ARG (no density),
 * ERR_NOT_CONVERGED (J - I numerically singular), ERR_OOM. */
xlbomd_status xlbomd_kernel_exact(xlbomd_ctx* ctx, int sys);

/* Energy monitor (row a10): the free-energy shadow potential
 * Omega[n](R) = U[n](R) - Te S[f] of Section IV.B (Eq. S_entropy for S, with
 * the occupations of the expansion) and the constant of motion of Section IV.C
 * (Eq. ShadowH1: kinetic energy + Omega), written to XLBOMD_ENERGY as
 * [Omega, 2 Tr[D H0], 1/2 sum (2q - n) gamma n, -2 kB Te S, kinetic, total,
 * repulsion].  Requires xlbomd_density on the same state; synchronises the
 * stream.  Errors: ERR_ARG (no density), ERR_CUDA. */
xlbomd_status xlbomd_energy(xlbomd_ctx* ctx, int sys);

/* a1-a10 for every system, nsteps times (Eqs. Integration, VRL_Damp).  The
 * systems of the context that share a padded orbital count advance in
 * lockstep: their expansions, chemical-potential chains and probe chains run
 * as grouped tensor-core launches over all of them (split precisions), with
 * one stream synchronisation per chemical-potential pass and per probe index
 * for the whole group; a padded size held by one system takes the one-system
 * step.  Every system follows exactly its one-system trajectory (same mu
 * search, Newton-Schulz plan and probes; bitwise the same results).  Errors:
 * ERR_DIVERGED (max |q - n| above diverge_tol for any system), and those of
 * xlbomd_density and xlbomd_kernel_update. */
xlbomd_status xlbomd_step(xlbomd_ctx* ctx, int nsteps);

/* Copy a quantity to host memory (synchronises the stream). */
xlbomd_status xlbomd_get(xlbomd_ctx* ctx, int sys, int what, double* host_out);

/* Overwrite a quantity from host memory (R, V, N, NHIST, MU). */
xlbomd_status xlbomd_set(xlbomd_ctx* ctx, int sys, int what, const double* host_in);

/* Sizes: natoms and padded orbital count of system sys. */
xlbomd_status xlbomd_sizes(xlbomd_ctx* ctx, int sys, int* natoms, int* n_orb, int* n_pad);

/* Diagnostics: one split-precision tensor-core product C = A B^T (n x n, n a
 * multiple of 128, prec FP16x3, BF16x3 or TF32x3; sym = 1: symmetric-output
 * mode with a symmetric B; sym = 2: the symmetric-output pair product
 * A B^T + B A^T; sym + 4: the same with one product of the hi operands only, as
 * in the single-product chains) of seeded uniform [-1, 1) matrices, compared on the
 * device with the FP64 product of the same FP64 inputs.  Other sym values:
 * ERR_ARG.  result[0] = max |C_tc - C_fp64|,
 * result[2] = device wait-timeout flag, result[3] = ms per product.
 * prec = XLBOMD_FP64 (sym 0 or 1) times one product of the plain-FP64 path
 * instead (result[3]; no comparison, result[0..2] = 0), synchronising the
 * device.  This is a check of the matrix-product engine; the paper has no
 * counterpart. */
xlbomd_status xlbomd_selftest_gemm(int n, int prec, int sym, double* result);

/* Diagnostics: the grouped product launch (the products of several systems of one size in
 * one persistent launch, per-problem tensor maps and epilogue arguments read from a device
 * table) against single launches: nprob (2..64) seeded operand pairs of size n, each product
 * computed alone, then all together in one grouped launch (both tile widths, as the tile
 * autotuner tries them, then the width it keeps).  sym as for xlbomd_selftest_gemm (0-2, +4
 * single product); prec FP16x3, BF16x3 or TF32x3.  result[0] = max |C_group - C_single| (0: the
 * grouped launch computes every tile exactly as the single launch does), result[1] = device
 * wait-timeout flag.  The paper has no counterpart. */
xlbomd_status xlbomd_selftest_gemm_group(int n, int prec, int sym, int nprob, double* result);

/* Diagnostics: number of CUDA kernels the library has launched since it was
 * loaded (all contexts). */
long long xlbomd_launch_count(void);

/* Diagnostics: CUDA-event timing of the matrix products of a context, taken
 * on the context's stream.  mode 1 = start (reset) recording, 0 = stop,
 * 2 = collect (synchronises) out[0] = products recorded, out[1] = their total
 * device time in ms, out[2] = their algorithmic flops (2 n^3, half for a
 * symmetric-output product).  The paper has no counterpart. */
xlbomd_status xlbomd_gemm_profile(xlbomd_ctx* ctx, int mode, double* out);

xlbomd_status xlbomd_clear_error(xlbomd_ctx* ctx);
const char* xlbomd_last_error(xlbomd_ctx* ctx);
xlbomd_status xlbomd_free(xlbomd_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* XLBOMD_API_H_ */
