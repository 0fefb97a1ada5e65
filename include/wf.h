/*
 * wf.h -- C ABI of libwf: the temporally preconditioned anisotropic Wilson operator
 * and its Krylov solve on one GPU (sm_103a), after B. Joo, R. G. Edwards and
 * M. J. Peardon, "An anisotropic preconditioning for the Wilson fermion matrix on
 * the lattice", arXiv 0910.0992.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Lattice: L^3 x T sites, spatially periodic; time boundary sign bc = +1 (periodic)
 *   or -1 (antiperiodic). L must be even and >= 2; 2 <= T <= 256.
 * Operator: the paper's Wilson matrix (§II, Eq. for M with A = 0)
 *       M = mu - D_t - D_s / gamma_f,   mu = 1 / (2 kappa_t),   gamma_f = kappa_t / kappa_s,
 *   i.e. 1/(2 kappa_t) times the hopping-parameter form; D_t and D_s are the temporal
 *   and spatial hopping terms with projectors (1 -+ gamma_mu)/2 (§II, Eqs. for D_t, D_s).
 * Spin basis: Euclidean Dirac-Pauli, gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],
 *   gamma_t = diag(1, 1, -1, -1), gamma_5 = gamma_x gamma_y gamma_z gamma_t; so P_+ = (1 + gamma_t)/2
 *   keeps spins 0-1 and P_- spins 2-3 (§II.C, "Dirac-Pauli spin basis").
 * Temporal wrap: T[N_t-1, 0] = -bc U_t(N_t-1) (§II.A; the printed form of this entry is
 *   garbled, this reading makes mu - D_t = C_L^-1 C_R^-1 hold).
 * Arrays (all complex128, interleaved re/im, C order):
 *   gauge   U[t][z][y][x][mu][row][col], mu = 0, 1, 2, 3 for x, y, z, t; links must be SU(3).
 *   spinor  psi[rhs][t][z][y][x][spin][colour]                 ("full field")
 *   half    psi[rhs][t][k][spin][colour], k the index of the site among the sites of one
 *           3-D parity p3 = (x + y + z) mod 2 in lexicographic order: k = (x >> 1) + (L/2)(y + L z)
 *           ("odd field" when p3 = 1).
 * Pointers: every array argument may be host or device memory of the handle's GPU; the library
 *   tells them apart (cudaPointerGetAttributes) and copies host arrays in and out itself; device
 *   memory of another GPU returns WF_EINVAL. A call reads every input in full into its own
 *   buffers before it writes any output, so an output may be the same array as an input (an
 *   in-place apply). The library never keeps a caller pointer after a call returns.
 * Streams: all device work is ordered on the handle's stream (wf_set_stream); every call
 *   returns only when its results are complete (calls are synchronous for status).
 * Errors: every int-returning call returns WF_OK or one of the codes below and records a
 *   message readable with wf_last_error. No C++ exception crosses the ABI.
 */
#ifndef WF_H
#define WF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wf_handle wf_handle_t;

enum wf_status {
  WF_OK = 0,
  WF_EINVAL = 1,     /* invalid argument: sizes, parameters, pointers, no gauge loaded */
  WF_ENOMEM = 2,     /* device allocation failed */
  WF_ECUDA = 3,      /* a CUDA runtime call failed */
  WF_ESINGULAR = 4,  /* the temporal preconditioner does not exist: det(1 - bc mu^-T P) ~ 0 */
  WF_ENOCONV = 5,    /* solver stopped at its iteration limit; outputs are still written */
  WF_ENAN = 6,       /* NaN or Inf met in a norm during a solve */
  WF_ETIMEOUT = 7    /* a bounded device-side wait expired (the opt-in TMA-fed kernels, WF_TMA=1) */
};

enum wf_method {
  WF_UNPREC = 0,         /* CGNR on M */
  WF_EO4D = 1,           /* CGNR on the 4-D Schur (even-odd) operator (§II.B, 4D-Schur) */
  WF_TEMPORAL = 2,       /* CGNR on C_L M C_R (§II.A) */
  WF_TEMPORAL_SCHUR = 3, /* CGNR on M-hat = 1 - gamma_f^-2 D-bar^oe D-bar^eo (§II.B, Eq. TPrecFull) */
  WF_TEMPORAL_ILU = 4    /* CGNR on M-tilde_ILU = S_L (M + A) S_R, the clover operator with partial temporal
                            preconditioning and 3-D ILU (§II.B, Eq. TPrecPartial; App. B) */
};

enum wf_precision {
  WF_FP64 = 0,    /* every operator apply in FP64 */
  WF_FP32 = 1,    /* FP32 operator applies; FP64 true residual. WF_TEMPORAL_SCHUR: defect
                     correction (FP32 S_L, CGNR and S_R per pass, see wf_solve); other methods, and
                     WF_TEMPORAL_SCHUR with environment WF_DC=0: FP64 reliable updates, S_L / S_R */
  WF_FP16MIX = 2  /* FP16-stored spinors with FP32 arithmetic in the CG (vectors and M-hat's
                     intermediate fields), FP32 reliable updates of the FP32 increment every 1e-2
                     drop (environment WF_RELIABLE_DELTA16), inside the defect-correction passes of
                     WF_FP32; with WF_DC=0 FP64 reliable updates every 1e-5 (WF_RELIABLE_DELTA) and
                     FP64 S_L / S_R instead; WF_TEMPORAL_SCHUR in the axial frame only */
};

#define WF_X0 1 /* wf_solve flag: x holds the initial guess on entry */
#define WF_MAX_SOLVE_RHS 1024 /* right-hand sides of one solve (all lattices of a joint wf_solve_many) */

/* Create a handle for an L^3 x T lattice (§II). kappa_t <= 0 selects kappa_t = xi * kappa_s.
 * bc = +1 or -1. Allocates the gauge storage on the current device. Returns WF_EINVAL for
 * odd or too small L, T outside [2, 256], kappa_s <= 0 or bc not +-1. Time lines longer than 128
 * sites run on the n-sites-per-lane kernels only (up to 8 sites per lane): FP64 and FP32 solves
 * and applies; FP16MIX, the one-thread-per-site and bulk-fed hop kernels and joint ragged solves
 * need T <= 128. */
int wf_create(int L, int T, double xi, double kappa_s, double kappa_t, int bc, wf_handle_t** out);

/* Host-only check (no GPU needed) of the index tables the kernels use for an L^3 x T lattice with
 * nrhs sources and traversal tiles of tile_rows rows of y (0: the default): the neighbour tables
 * of both parities (every entry a line of the other parity whose opposite neighbour is the entry's
 * line), the traversal order (every (source, line) pair once) and the bulk-fed kernels' units
 * (every (source group, line) pair once, for groups of 1 and 2). The library runs the same checks
 * whenever it builds a table. plant = 1, 2 or 3 corrupts one entry of the neighbour, traversal or
 * unit table after it is built (a self-test of the checks). Returns WF_OK, WF_EINVAL for invalid
 * arguments (tile_rows not dividing L), or WF_ECUDA if a check failed. */
int wf_check_tables(int L, int T, int nrhs, int tile_rows, int plant);

/* Release the handle and all its device memory. Null is accepted. */
int wf_destroy(wf_handle_t* h);

/* Order all later device work of h on this CUDA stream (a cudaStream_t; 0 = legacy default). */
int wf_set_stream(wf_handle_t* h, void* stream);

/* Message of the last error on h (never null; empty after success). */
const char* wf_last_error(const wf_handle_t* h);

/* Choose the frame the library works in, before wf_load_gauge (a later call discards the loaded
 * field). axial = 1 (the default): at load the field is rotated, per time line, to the axial
 * (temporal) gauge, U_t(t) = 1 for t < T-1 and U_t(T-1) = P the Polyakov product (§II.C,
 * "axial gauge"; App. C), so T^-1 needs no U_t and no 3x3 products; inputs and outputs are
 * rotated in and out, so every result is the same as in the caller's gauge. axial = 0: the
 * field is used as given and T^-1 composes 3x3 affine maps along each line. */
int wf_set_gauge_frame(wf_handle_t* h, int axial);

/* Sizes of the arrays the handle works on: complex128 elements per right-hand side. */
long long wf_field_elems(const wf_handle_t* h);  /* full field: 12 L^3 T */
long long wf_half_elems(const wf_handle_t* h);   /* one parity: 6 L^3 T  */

/* Load a gauge field (layout above). The library copies it (FP64 master, FP32 shadow, links
 * split into U_t and spatial links by 3-D parity) and builds, per spatial site, the SMW
 * wrap-around matrices Lambda = (1 - bc mu^-T P)^-1 of T^-1 and its counterpart for T^-dag
 * (§II.A, step 1: X(0) = -bc mu^-T P with P the Polyakov product, Lambda = (I + W^dag X)^-1).
 * Returns WF_EINVAL, with nothing loaded, if an entry is NaN or Inf or a link is not SU(3)
 * within 1e-9 (largest entry of U^dag U - 1 and |det U - 1|: the FP32 storage keeps two rows
 * of each link and rebuilds the third, which needs det U = 1), and WF_ESINGULAR if some
 * |det(1 - bc mu^-T P)| < 1e-12. */
int wf_load_gauge(wf_handle_t* h, const double* U);

/* out = M in (dagger = 0) or M^dag in = gamma_5 M gamma_5 in (dagger = 1); full fields, nrhs of
 * them back to back (§II, Eq. for M). */
int wf_apply_M(wf_handle_t* h, const double* in, double* out, int dagger, int nrhs);

/* out = T^-1 in (dagger = 0) or (T^dag)^-1 in (dagger = 1) on every spin component of full
 * fields: the exact inverse of the cyclic temporal matrix of every spatial site (§II.A, Eq. for T
 * and the SMW inverse). */
int wf_apply_Tinv(wf_handle_t* h, const double* in, double* out, int dagger, int nrhs);

/* out = C_L in = (P_+ + P_- T^-1) in (which = 0) or C_R in = (P_- + P_+ T^-dag) in (which = 1),
 * full fields (§II.A). */
int wf_apply_C(wf_handle_t* h, const double* in, double* out, int which, int nrhs);

/* out_odd = M-hat in_odd (dagger = 0) or M-hat^dag in_odd = gamma_5 M-hat gamma_5 in_odd
 * (dagger = 1) on odd fields, where (§II.B, Eq. TPrecFull and the D-bar definition)
 *   M-hat = 1 - gamma_f^-2 C_L^o D_s^oe C_R^e C_L^e D_s^eo C_R^o. */
int wf_apply_schur(wf_handle_t* h, const double* in_odd, double* out_odd, int dagger, int nrhs);

/* The comparator of the paper's preconditioner: out = M-hat_4 in (dagger = 0) or gamma_5 M-hat_4
 * gamma_5 in (dagger = 1), the standard 4-D even-odd Schur operator
 *   M-hat_4 = mu - mu^-1 D_w^oe D_w^eo,   D_w = D_t + D_s / gamma_f   (§II.B, 4D-Schur; App. B),
 * on arrays of the sites with (x + y + z + t) odd, in lexicographic order: [rhs][V/2][spin][colour],
 * site k = (x + L (y + L (z + L t))) / 2. Needs an even T. */
int wf_apply_eo4d(wf_handle_t* h, const double* in_odd4, double* out_odd4, int dagger, int nrhs);

/* FP32 variants: same contracts, FP64 in and out, every internal step in FP32. */
int wf_apply_eo4d_f32(wf_handle_t* h, const double* in_odd4, double* out_odd4, int dagger, int nrhs);
int wf_apply_M_f32(wf_handle_t* h, const double* in, double* out, int dagger, int nrhs);
int wf_apply_Tinv_f32(wf_handle_t* h, const double* in, double* out, int dagger, int nrhs);
int wf_apply_schur_f32(wf_handle_t* h, const double* in_odd, double* out_odd, int dagger, int nrhs);
/* M-hat with FP16-stored fields and FP32 arithmetic, the operator of the WF_FP16MIX solve (north-
 * star precision pattern; the paper fixes no precision): each source is stored divided by its RMS,
 * so results carry FP16 rounding (about 1e-3 relative) for inputs of any range. Axial frame only;
 * WF_EINVAL for lattices the one-thread-per-site kernels do not serve. */
int wf_apply_schur_f16(wf_handle_t* h, const double* in_odd, double* out_odd, int dagger, int nrhs);

/* Solve M x = rhs for nrhs full-field right-hand sides with CG on the normal equations of the
 * operator `method` selects, FP64 or mixed `precision`. For WF_TEMPORAL_SCHUR the source is
 * prepared with S_L and the solution recovered with S_R (§II.B, S_L and S_R). A solve is done
 * when the FP64 true residual ||rhs - M x||_2 / ||rhs||_2 <= tol, computed with the full M.
 * iters_out[k] (CG iterations) and true_resid_out[k] are written for every right-hand side
 * (host arrays of nrhs entries; either may be null). flags: WF_X0 to start from x.
 * 1 <= nrhs <= WF_MAX_SOLVE_RHS (else WF_EINVAL).
 * WF_FP32 with WF_TEMPORAL_SCHUR: defect correction. Each pass solves M d = r entirely in FP32
 * (S_L, CGNR on M-hat, S_R) to a 1e-5 reduction of its residual (environment WF_DC_RHO), adds d
 * to the FP64 solution and recomputes the FP64 true residual r = rhs - M x; two passes reach
 * 1e-10 on the benchmark lattices. Environment WF_DC=0 selects the scheme of the other methods.
 * WF_FP32 with the other methods: FP32 CG iterations whose residual is recomputed in FP64
 * whenever it fell by 1e-5 (reliable updates; environment WF_RELIABLE_DELTA).
 * CG iterations run in blocks whose convergence checks happen on the device, one iteration
 * replayed as a CUDA graph when the handle has a stream of its own (environment WF_GRAPH=0: plain
 * launches). The first FP32 solve or apply for a given nrhs also tunes the Schur operator's
 * kernels (see wf_hop_config).
 * Returns WF_ENOCONV (outputs written: the last iterate) if some right-hand side missed tol
 * within the handle's iteration limit (wf_set_max_iterations), WF_ENAN if a norm became NaN or
 * Inf (a NaN or Inf in rhs or x0 ends the solve this way). */
int wf_solve(wf_handle_t* h, const double* rhs, double* x, int nrhs, double tol, int method, int precision,
             int flags, int* iters_out, double* true_resid_out);

/* Several solves in one call (ragged batches, such as a sweep over lattice sizes at one
 * anisotropy): handle hs[i] (one lattice each, possibly of different sizes; the handles must be
 * distinct) solves nrhs[i] sources rhs[i] into x[i], with the arguments and conventions of wf_solve
 * (tol, method, precision and flags common to all).
 *   - Default: every solve runs on a host thread of its own and on its handle's stream (a
 *     temporary stream for handles on the default stream), so that the lattices' solves overlap on
 *     the GPU, each in its own phase (one lattice's FP64 true residual beside another's FP32
 *     iterations).
 *   - Joint path (environment WF_JOINT=1): FP32 temporal + Schur solves (WF_TEMPORAL_SCHUR,
 *     WF_FP32, defect correction) on handles of one device, in the axial frame, with one iteration
 *     limit, no clover term and at most WF_MAX_SOLVE_RHS sources in all are solved as one CGNR per
 *     defect-correction pass over the concatenation of all lattices' sources. Each of its kernels
 *     (K-a, K-b, K-c, the vector updates, norms and convergence checks) runs as one launch over
 *     every lattice (eight lattices per launch at most; lattices grouped by kernel family and line
 *     length, bulk-fed ones on launches of their own) with the lattices' autotuned configurations
 *     (tuned in the call for a handle with none for its nrhs); S_L, the reconstruction and the FP64
 *     true residual run per lattice, each on its handle's stream. Every source keeps its own CG
 *     scalars and stopping test, so it takes the iterations of a separate solve (up to the rounding
 *     of its norms). The call first synchronises every handle's stream; the iterations run on
 *     hs[0]'s stream; a handle on the default stream, or on a stream another handle uses, works on
 *     a temporary stream. An error is reported on every handle and as every status. Measured on
 *     GB300 it is 10-25 % slower than the default, whose overlapping phases it gives up.
 * No counterpart in the paper (its solves are independent problems). iters_out, resid_out and
 * status_out may be null, or hold n pointers (n statuses); returns WF_OK or the first non-OK
 * status. */
int wf_solve_many(int n, wf_handle_t* const* hs, const double* const* rhs, double* const* x, const int* nrhs,
                  double tol, int method, int precision, int flags, int* const* iters_out,
                  double* const* resid_out, int* status_out);

/* The FP64 M-hat apply of wf_apply_schur, with every byte of its work memory taken from one
 * fixed device array that the library reserves, so this call allocates nothing. For callers
 * that cannot have a library call cudaMalloc at apply time: applications whose own pool has
 * reserved nearly all device memory, latency-critical loops (cudaFree synchronises the device),
 * processes with a device-memory budget fixed at start-up. The paper has no counterpart; it is
 * a deployment variant of the same operation.
 *   - in_odd and out_odd must be device memory of the handle's GPU (odd fields as for
 *     wf_apply_schur); host memory or another GPU's memory returns WF_EINVAL.
 *   - Work memory: WF_NOALLOC_SCRATCH_BYTES per device; it holds 4 internal odd fields of
 *     nrhs right-hand sides, so roughly nrhs * L^3 * T <= 43,000 sites (e.g. 8^3 x 64 or
 *     12^3 x 24 for nrhs = 1). Larger requests return WF_EINVAL with the size needed.
 *   - The array exists on every GPU where the library's code is loaded and stays allocated
 *     until the process exits. Every call looks up its device address in the current context
 *     (cudaGetSymbolAddress) with the handle's device current.
 *   - The call returns after its work has finished (it synchronises the handle's stream).
 *   - All calls on a device share the array; each call clears what it uses first. Calls whose
 *     device work overlaps (several streams, handles or host threads) race: order them. */
#define WF_NOALLOC_SCRATCH_BYTES (16u << 20)
int wf_apply_schur_noalloc(wf_handle_t* h, const double* in_odd, double* out_odd, int dagger, int nrhs);

/* Clover (SW) operator M_SW = A + mu - D_t - D_s / gamma_f (§II, Eq. for M and for A), with
 *   A(x) = -[(c_t/2) sum_i sigma_i0 F_i0(x) + (c_s/2) sum_{i<j} sigma_ij F_ij(x)],
 *   sigma_mu nu = [gamma_mu, gamma_nu] / 2 (Dirac-Pauli basis),
 *   F_mu nu = (Q_mu nu - Q_mu nu^dag) / 8 with its trace removed, Q_mu nu(x) the sum of the four
 *   plaquette leaves of the mu nu plane at x (orientation of U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag).
 * c_s and c_t are the caller's (Eq. ClovCoeffs gives their tadpole-improved values).
 * wf_load_gauge_clover: wf_load_gauge(h, U), then A built from the same U (FP64, stored with an
 * FP32 copy, 2 x 36 complex per site; for even T also the blocks of mu + A and (mu + A)^-1 in the
 * 4-D even-odd layout, WF_ESINGULAR if some block has no inverse); a later wf_load_gauge removes
 * it. While a clover term is loaded, wf_solve accepts WF_TEMPORAL_ILU and WF_EO4D, which then
 * solve M_SW, WF_EO4D with the 4-D Schur clover operator (mu + A)^oo - D_w^oe (mu + A)^-1_ee D_w^eo
 * (§II.B, the paper's comparator), which wf_apply_eo4d then applies; wf_force returns WF_EINVAL
 * and the other apply entry points keep applying the Wilson operators.
 * wf_apply_clover: out = A in on full fields [rhs][V][spin][colour] (FP64).
 * wf_apply_ilu: out = M-tilde_ILU in (dagger: gamma_5 M-tilde_ILU gamma_5) on full fields, with
 *   M-tilde_ILU = S_L M_SW S_R (the Wilson S_L, S_R of §II.B applied to M_SW), applied by the
 *   sequence of App. B: t1 = g Dbar^eo psi_o, t2 = Abar^ee (t1 + psi_e), chi_e = psi_e + t2,
 *   chi_o = psi_o + Abar^oo psi_o + g Dbar^oe (t2 - t1), g = 1/gamma_f, Abar = C_L A C_R,
 *   Dbar = C_L D_s C_R; without a clover term A = 0 and it is diag(1, M-hat). _f32: FP32 steps.
 * wf_solve(..., WF_TEMPORAL_ILU, ...) solves M_SW x = rhs as M-tilde_ILU y = S_L rhs, x = S_R y,
 * accepted on the FP64 true residual of M_SW; no initial guess (WF_X0 gives WF_EINVAL).
 * Errors: WF_EINVAL (no gauge field; no clover term for wf_apply_clover; non-finite c_s, c_t). */
int wf_load_gauge_clover(wf_handle_t* h, const double* U, double c_s, double c_t);
int wf_apply_clover(wf_handle_t* h, const double* in, double* out, int nrhs);
int wf_apply_ilu(wf_handle_t* h, const double* in, double* out, int dagger, int nrhs);
int wf_apply_ilu_f32(wf_handle_t* h, const double* in, double* out, int dagger, int nrhs);

/* Full SW temporal preconditioning (§II.A, the paragraphs on SW fermions; appendix "Full
 * Preconditioning with Clover"): the whole temporal block Q = A + mu - D_t of every spatial line,
 * clover term included, is inverted, and the 3-D Schur operator on odd sites is
 *   M-hat_full = 1 - gamma_f^-2 (Q^oo)^-1 D_s^oe (Q^ee)^-1 D_s^eo
 * (Eq. TPrecFull with C_L = Q^-1, C_R = 1). A is the term of wf_load_gauge_clover, or 0 if none is
 * loaded (then Q = mu - D_t = C_L^-1 C_R^-1). Q^-1 is the appendix's single Woodbury step
 * Q = T_0 + V W^dag around the open chain T_0, which the library factors by block LU instead of
 * the paper's inner CG, in the precision of the call: the blocks Sigma_t^-1 and the Woodbury
 * columns T_0^-1 V, 4.6 KB of device memory per site in FP64, 2.3 KB in FP32. The factors are kept
 * for later calls; every call first compares a 64-bit fingerprint of the arrays they were formed
 * from (clover term, U_t or P, frame) with the current ones and factors again on a change.
 * wf_apply_Qinv: out = Q^-1 in on full fields [rhs][V][spin][colour]; _f32: FP32 applies.
 * wf_apply_schur_full_sw: out = M-hat_full in (dagger: its adjoint) on odd fields as for
 *   wf_apply_schur; _f32: FP32 arithmetic.
 * wf_solve_full_sw: M_SW x = rhs (M_SW = M + A) on full fields by CGNR on M-hat_full with
 *   b = (Q^oo)^-1 (rhs_o + gamma_f^-1 D_s^oe (Q^ee)^-1 rhs_e) and x_e = (Q^ee)^-1 (rhs_e +
 *   gamma_f^-1 D_s^eo x_o), in defect-correction passes (at most 8) that each solve for the FP64
 *   true residual r = rhs - M_SW x in `precision` (WF_FP64, or WF_FP32 with passes to 1e-5) and add
 *   the correction in FP64, until |r_k| <= tol |rhs_k| for every right-hand side; the handle's
 *   iteration limit bounds all passes together. iters_out[k] (CG iterations of right-hand side k)
 *   and true_resid_out[k] (host, may be null) are written for every k.
 * Arrays follow the conventions above (host or device memory; in-place calls allowed). Errors: WF_EINVAL (no gauge field, nrhs outside [1, WF_MAX_SOLVE_RHS], tol <= 0,
 * precision other than WF_FP64 / WF_FP32), WF_ESINGULAR (a block of the factorisation, or the
 * 12x12 Woodbury matrix of a line, has no inverse), WF_ENAN (a non-finite norm in the solve),
 * WF_ENOCONV (iteration limit or 8 passes reached; x holds the last iterate). */
int wf_apply_Qinv(wf_handle_t* h, const double* in, double* out, int nrhs);
int wf_apply_Qinv_f32(wf_handle_t* h, const double* in, double* out, int nrhs);
int wf_apply_schur_full_sw(wf_handle_t* h, const double* in_odd, double* out_odd, int dagger, int nrhs);
int wf_apply_schur_full_sw_f32(wf_handle_t* h, const double* in_odd, double* out_odd, int dagger, int nrhs);
int wf_solve_full_sw(wf_handle_t* h, const double* rhs, double* x, int nrhs, double tol, int precision,
                     int* iters_out, double* true_resid_out);

/* Pseudofermion force of the temporally preconditioned operator. For the action
 *   S = phi^dag (M-hat^dag M-hat)^-1 phi,   phi an odd field (as for wf_apply_schur, one source),
 * writes F[t][z][y][x][mu][a] (real, 8 per link, mu = x, y, z, t) = dS/d eps for the perturbation
 * U_mu(x) -> exp(i eps T_a) U_mu(x), T_a = lambda_a / 2 (the Gell-Mann matrices halved), in the
 * caller's gauge. X = (M-hat^dag M-hat)^-1 phi by CG to |phi - M-hat^dag M-hat X| <= tol |phi|
 * (precision: FP64, or FP32 iterations with FP64 reliable updates); then, with Y = M-hat X,
 * dS = -2 Re(Y^dag dM-hat X) summed over the six factors of M-hat (§II.B), all in FP64. The
 * paper proposes the HMC use of the preconditioner without working it out (§IV). action (host,
 * may be null) receives S = |Y|^2; iters (host, may be null) the CG iterations. F may be host
 * or device memory, or null to compute the action alone. */
int wf_force(wf_handle_t* h, const double* phi_odd, double* F, int precision, double tol, double* action,
             int* iters);

/* Determinant of the temporal preconditioner, the extra Hamiltonian term of hybrid Monte Carlo
 * with the preconditioned operator (the paper anticipates such terms in §IV without deriving
 * them). C_L^-1 C_R^-1 = mu - D_t (§II.A) and the 3-D Schur complement of C_L M C_R is M-hat
 * (§II.B), so det M = det(M-hat) det(mu - D_t), and per spatial line det T = det(mu^N_t - s P)
 * with P = U_t(0) ... U_t(N_t - 1), so
 *   logdet = log det(mu - D_t) = 4 sum_x log|det(mu^N_t - s P(x))|   (real: det(mu - D_t) >= 0).
 * Two flavours carry -2 logdet in their action beside phi^dag (M-hat^dag M-hat)^-1 phi.
 * F (may be null; host or device memory) receives F[t][z][y][x][mu][a] = d logdet / d eps for
 * U_mu(x) -> exp(i eps T_a) U_mu(x), T_a = lambda_a / 2, in the caller's gauge: 8 reals per link,
 * zero for the spatial links (layout as for wf_force). logdet (host, may be null) receives the
 * value. All in FP64 from the loaded gauge field. WF_EINVAL if no gauge field is loaded. */
int wf_temporal_logdet(wf_handle_t* h, double* logdet, double* F);

/* Autotuned configuration of the FP32 hop kernels of M-hat (no counterpart in the paper): the
 * first FP32 Schur apply of a handle for a given nrhs times every candidate and keeps the fastest
 * (environment WF_AUTOTUNE=0 at the first apply keeps the built-in choice; WF_HOP fixes one, see
 * the README). variant: 1 one thread per site, 2 n sites per lane, 3 bulk-copy-fed (shared-memory
 * stages filled by cp.async.bulk); tile_rows: rows of y per traversal tile; ms: the chosen
 * candidate's K-b + K-c time over three runs (0 if fixed by WF_HOP). wf_hop_pipe_config gives the
 * bulk-fed kernels' sources per unit (1 or 2) and stages (2 to 4); both are 0 for variants 1 and 2.
 * Any output pointer may be null. WF_EINVAL if that nrhs has not been tuned (yet). */
int wf_hop_config(wf_handle_t* h, int nrhs, int* variant, int* tile_rows, float* ms);
int wf_hop_pipe_config(wf_handle_t* h, int nrhs, int* sources_per_unit, int* stages);

/* CG iteration limit of every later solve and force on h (no counterpart in the paper; for a
 * defect-correction solve the iterations of all its passes together): maxiter >= 1, or 0 for the
 * default 100000. WF_EINVAL if maxiter < 0. */
int wf_set_max_iterations(wf_handle_t* h, int maxiter);

/* Number of kernels this handle has launched since it was created (all entry points). */
long long wf_launch_count(const wf_handle_t* h);

/* Per-kernel timing on the handle's stream (CUDA events around every launch), for
 * benchmarks. wf_profile(h, 1) clears the counters and starts recording; wf_profile(h, 0)
 * stops. wf_profile_get fills up to cap entries of (name, launches, total milliseconds) and
 * returns how many kernels were recorded. Names stay valid while h lives. */
int wf_profile(wf_handle_t* h, int on);
int wf_profile_get(wf_handle_t* h, const char** names, long long* launches, double* total_ms, int cap);

#ifdef __cplusplus
}
#endif

#endif /* WF_H */
