/*
 * helm_dd.h -- C ABI of a GB300 (sm_103a) solver for the 2-D/3-D Helmholtz
 * equation  -Lap u - k^2 u = f,  k = omega / c,  truncated by a PML, with the
 * double-sweep PML-transmission preconditioner of
 *
 *   C. C. Stolk, "A rapidly converging domain decomposition method for the
 *   Helmholtz equation", arXiv:1208.3956  (Sections 2.1-2.3, Algorithms 1-5).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid.      The interior grid has n[0] x n[1] (x n[2]) points with spacing h.
 *            A PML of w_outer points is added outside it on every side, so the
 *            padded grid has N[a] = n[a] + 2*w_outer points per axis.  The speed
 *            is clamp-extended into the added layer.
 * Fields.    rhs / u / in / out are complex128 arrays on the PADDED grid,
 *            interleaved (re, im) doubles, x fastest, one right-hand side after
 *            another: element (b, z, y, x) sits at complex offset
 *            ((b*N[2] + z)*N[1] + y)*N[0] + x   (N[2] = 1 in 2-D).
 *            Speeds c and gradients are real doubles on the INTERIOR grid, x
 *            fastest.
 * Pointers.  Every array argument may be a host pointer or a CUDA device pointer
 *            (detected per call).  Host arrays are copied in and out inside the
 *            call.  Buffers are borrowed for the duration of the call only.
 *            Device complex128 fields must be 16-byte aligned (HELM_EINVAL
 *            otherwise: the kernels read them with 16-byte accesses).
 * Sync.      Calls are synchronous on return.  A handle is not thread-safe;
 *            separate handles are independent.
 * Errors.    Every call returns a helm_status and never aborts or throws across
 *            the ABI.  helm_dd_last_error() gives a human-readable reason for the
 *            last failure on a handle.
 * Operator.  A is the paper-form finite-difference operator of Section 2.2
 *            (5-point in 2-D, 7-point in 3-D; inside a layer
 *            alpha(x_i)[alpha(x_{i+1/2})(u_{i+1}-u_i) - alpha(x_{i-1/2})(u_i-u_{i-1})]/h^2
 *            with alpha = 1/(1 + i sigma/omega)); u = 0 one point beyond the
 *            padded grid.  The PML profile is sigma(d) = sigma0 (d/L)^2 with
 *            L = w*h and sigma0 = 3 c_ref ln(1e6) / (2L); c_ref defaults to the
 *            maximum of c.
 */
#ifndef HELM_DD_H
#define HELM_DD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct helm_dd helm_dd;   /* opaque; owns all device memory it allocates */

typedef enum {
    HELM_OK = 0,
    HELM_EINVAL = -1,     /* invalid argument (sizes, c <= 0 or NaN, omega <= 0, ...) */
    HELM_ENOMEM = -2,     /* device allocation failed                                 */
    HELM_ECUDA = -3,      /* a CUDA call failed                                       */
    HELM_ESTATE = -4,     /* call out of order (e.g. apply before factor)            */
    HELM_ENOTCONV = -5,   /* GMRES hit maxit; the best iterate and info are written   */
    HELM_ENUMERIC = -6,   /* tiny pivot in a block inverse, or NaN/Inf in a norm      */
    HELM_ETIMEOUT = -7    /* a bounded device wait gave up                            */
} helm_status;

typedef struct {
    int dim;          /* 2 or 3                                        */
    int64_t n[3];     /* interior points per axis (x, y, z); n[2]=1 in 2-D */
    double h;         /* grid spacing                                  */
} helm_grid;

typedef enum {
    HELM_PREC_FP64 = 0,   /* complex128 factors and sweeps, FP64 GMRES                  */
    HELM_PREC_MIXED = 1   /* complex64 factors and sweeps (FP32 accumulate), FP64 FGMRES */
} helm_prec;

typedef enum {
    HELM_TRANSMISSION_PML = 0,    /* added PML layers, single-layer transfers (Section 2.1)  */
    HELM_TRANSMISSION_ROBIN = 1   /* Robin transmission conditions (Section 4.4)           */
} helm_transmission;

typedef enum {
    HELM_SWEEP_DOUBLE = 0,        /* forward sweep, residual, backward sweep (Section 2.1)   */
    HELM_SWEEP_CONCURRENT = 1     /* upward and downward sequences at once (Sections 1.2, 3.1) */
} helm_sweep;

typedef struct {
    int iters;        /* Arnoldi steps (= preconditioner applications in the Krylov loop) */
    double rel_res;   /* true final ||f - A u||_2 / ||f||_2 over the padded grid           */
    double t_ms;      /* wall time of the whole batch solve                               */
} helm_rhs_info;

/* Create a problem on the padded grid and validate its parameters
 * (Section 2.1: strips D^(j) along x with J subdomains; Eq. define_beta_j,
 * read as an even split of the interior: beta_j = w_outer-1 + floor(j n_x/J + 1/2),
 * the first and last strips also owning the outer layer).
 *   g        grid; dim 2 or 3, n[a] >= 1, h > 0
 *   c        speed on the interior grid (x fastest), all finite and > 0; copied
 *   omega    angular frequency > 0
 *   w_outer  outer PML width in points (>= 0)
 *   w_sub    added PML width of each strip on its internal sides (>= 1 if J > 1)
 *   J        number of strips (>= 1); every strip core must have >= 2 columns
 *   prec     arithmetic of factors and sweeps
 *   out      receives the handle (NULL on failure)
 * Returns HELM_EINVAL on bad arguments, HELM_ENOMEM / HELM_ECUDA on device errors. */
helm_status helm_dd_create(const helm_grid* g, const double* c, double omega,
                           int w_outer, int w_sub, int J, helm_prec prec, helm_dd** out);

/* Fix the speed c_ref that sets the PML strength sigma0 (default: max of c).
 * Must be called before helm_dd_factor; c_ref > 0. */
helm_status helm_dd_set_pml_speed(helm_dd* h, double c_ref);

/* Number of chunks P the y-axis of every strip is cut into for the partitioned
 * block-tridiagonal factorisation (1 = plain sequential block LU).  0 selects the
 * built-in choice: about 0.93 N_y^(2/3), lowered when a panel of more than 4
 * right-hand sides is set before helm_dd_factor (helm_dd_set_panel) so that the
 * panel's tiles of 4 fit one wave of the SMs.  Must be called before helm_dd_factor. */
helm_status helm_dd_set_chunks(helm_dd* h, int P);

/* Number of groups G the P-1 separator rows of every strip are cut into (a
 * second level of nested dissection along y): G-1 separators become level-2
 * separators and the rest form G groups of consecutive separators, each solved
 * on its own before the small level-2 system couples them.  1 = one separator
 * chain; 0 selects the built-in choice (about sqrt(P-1)); values above P/2 are
 * clamped.  Must be called before helm_dd_factor.  The result is the same up to
 * rounding for every G. */
helm_status helm_dd_set_sep_groups(helm_dd* h, int G);

/* G in use after helm_dd_factor (0 before). */
int helm_dd_sep_groups(const helm_dd* h);

/* P in use after helm_dd_factor (0 before). */
int helm_dd_chunks(const helm_dd* h);

/* Most right-hand sides per internal panel of helm_dd_solve, helm_dd_solve_reduced
 * and helm_dd_gradient (the batching of many-source runs, not the paper's own
 * parameter): a call with more right-hand sides runs them panel after panel, so
 * that the Krylov basis (2 restart + 2 complex128 fields per right-hand side in
 * the full space) and the sweep buffers are held for one panel only.  A panel is
 * never wider than the free device memory holds; 0 (the default) sets no other
 * cap.  Results do not depend on the panel width beyond rounding.  Set before
 * helm_dd_factor, a width above 4 also lowers the built-in chunk count
 * (helm_dd_set_chunks); after it, only the cap changes. */
helm_status helm_dd_set_panel(helm_dd* h, int nrhs);

/* Order of the strip solves of P (before helm_dd_factor; default HELM_SWEEP_DOUBLE).
 * HELM_SWEEP_CONCURRENT performs the upward and downward sequences simultaneously
 * (Section 1.2, "Results"; Section 3.1 states it for 1-D): an upward sequence v^(j)
 * on f (Eq. solve_upward) and a downward sequence y^(j) on f (Eq. solve_downward with
 * f in place of the residual g) run side by side on three streams; strip j's total
 * field u^(j) -- f on its physical columns plus the transfers from v^(j-1) and
 * y^(j+1) -- is v^(j) plus one more strip solve, and P f = u^(j) on D^(j).  It is
 * exact with perfect layers, like the double sweep, has about half its sequential
 * depth (J strip solves against 2J-1) and 3J-2 solves in all; the built-in chunk
 * count is capped at a third of the SMs so that three strip solves fit side by side.
 * PML transmission and 2-D grids only (HELM_EINVAL otherwise). */
helm_status helm_dd_set_sweep(helm_dd* h, helm_sweep mode);

/* Transmission condition of the double sweep (before helm_dd_factor; default PML).
 * HELM_TRANSMISSION_ROBIN is the comparison method of Section 4.4: the strips keep
 * their physical columns beta_{j-1}+1 .. beta_j+1 (an overlap of one column) but
 * carry no added PML (w_sub is ignored); at the half point beyond an internal
 * boundary column the condition -+d_x u + ik u = data holds, discretised as
 * a u_in + b u_out with a = 1/h + ik/2, b = -1/h + ik/2 (d_x u one-sided over the
 * half point, u the mean of the two values, k at the boundary column), the ghost
 * value eliminated into the strip operator.  The right sweep passes
 * d_x v^(j-1) + ik v^(j-1) at l^(j), the left sweep (on the residual g)
 * -d_x w^(j+1) + ik w^(j+1) at r^(j); the outer PML stays on the outer boundary.
 * 2-D grids only (helm_dd_factor returns HELM_EINVAL in 3-D). */
helm_status helm_dd_set_transmission(helm_dd* h, helm_transmission t);

/* Algorithm 1 (preparation): assemble every strip operator A^(j) on the grid of
 * Eq. grid_A_j (physical columns beta_{j-1}+1 .. beta_j+1 plus w_sub added PML
 * columns on internal sides, k held constant in x across an added layer) in its
 * complex-symmetric form S^(j) A^(j), and factor it as a block-tridiagonal
 * matrix along y.  Factors stay on the device.  Returns HELM_ENUMERIC on a
 * numerically singular block.
 * 2-D grids: W x W blocks, partitioned along y (nested dissection) for the
 * parallel sweep; a strip solve keeps a ring of at least four blocks in shared
 * memory, so HELM_EINVAL when a strip is too wide for it (complex128: about 50
 * columns; complex64: 64).  3-D grids: one dense block of n = W N_z unknowns (a slab of
 * W x-columns by all z-planes) per grid row y, factored top down with every
 * block inverted by Gauss-Jordan elimination with partial pivoting (complex64:
 * blocked, the updates on the tensor cores, the panels on thread-block clusters;
 * complex128: one cooperative launch per block); the strip solves of the sweep
 * run as cooperative launches (all CTAs co-resident), and a bounded wait inside
 * any of these kernels that gives up returns
 * HELM_ETIMEOUT.  HELM_EINVAL when a 3-D block exceeds 4096 unknowns in complex64
 * or 2048 in complex128 (use more strips).  Factor memory: N_y n^2 complex entries
 * per strip (8 or 16 bytes). */
helm_status helm_dd_factor(helm_dd* h);

/* out = P in for nrhs right-hand sides (Section 2.1, Eqs. solve_upward and
 * solve_downward; Algorithm 4 without u~): forward sweep j = 1..J with the
 * single-layer-potential transfer -2 delta(x-b_{j-1}) d_x v^(j-1), residual
 * g = f - A v, backward sweep j = J-1..1 with +2 delta(x-b~_j) d_x w^(j+1) on
 * g restricted to D~^(j), and out = v + w.  HELM_ESTATE before helm_dd_factor. */
helm_status helm_dd_apply_precond(helm_dd* h, const double* in, double* out, int nrhs);

/* out = P in, exactly as helm_dd_apply_precond, without allocating device memory.
 * The paper has no counterpart: this exists for callers that must not have the
 * library allocate while they run -- programs whose own pool allocator owns all
 * device memory, programs near the memory limit where a late workspace
 * allocation could fail, and latency-critical loops where cudaMalloc/cudaFree
 * would stall the device.  The work buffers come from one 64 MiB file-scope
 * device array.  The array (and every kernel module the call launches) is
 * loaded onto a device, and its 64 MiB taken, when a handle first uses that
 * device (in helm_dd_factor, with the handle's other device memory); its
 * device address is looked up there too, once per device with that device
 * current.  It is held until the process exits.  The call itself allocates
 * nothing.
 *   in, out   DEVICE pointers (complex128 fields as above), distinct; host
 *             pointers are rejected because staging them would allocate
 *   nrhs      number of fields; HELM_EINVAL (with the byte count in
 *             helm_dd_last_error) when 2*nrhs*N*16 bytes plus the strip
 *             buffers exceed the 64 MiB limit
 * All calls share the one array and each reuses what the previous call left
 * there, so calls that overlap on the GPU (other threads, other handles,
 * other streams) race and must be serialised by the caller.
 * HELM_ESTATE before helm_dd_factor. */
helm_status helm_dd_apply_precond_noalloc(helm_dd* h, const double* in, double* out, int nrhs);

/* out = A in (paper form, FP64) for nrhs fields. */
helm_status helm_dd_matvec(helm_dd* h, const double* in, double* out, int nrhs);

/* Solve A u = rhs for nrhs right-hand sides (Algorithm 5, full-space form):
 * right-preconditioned GMRES(restart) on A P v = f, u = P v (flexible form in
 * mixed precision), x0 = 0, stopping when the Givens estimate reaches
 * tol*||f|| and the true residual confirms it.  info (nrhs entries, may be NULL)
 * receives per-RHS iterations, true relative residual and the batch time.
 * Returns HELM_ENOTCONV (with u and info written) when maxit is reached. */
helm_status helm_dd_solve(helm_dd* h, const double* rhs, double* u, int nrhs,
                          double tol, int restart, int maxit, helm_rhs_info* info);

/* ---- The reduced space (Section 2.3, "Algorithm"; Algorithms 2-5).
 * Since f - A P f vanishes off the 2(J-1) grid lines x = beta_j+1, beta_j+2
 * (j = 1..J-1), GMRES can run on fields given on those lines only.  A reduced
 * array holds, per right-hand side, N[2] N[1] rows of L = 2(J-1) complex128
 * values, interleaved: element (b, z, y, i) sits at complex offset
 * ((b*N[2] + z)*N[1] + y)*L + i and is the field at padded column cols[i] of
 * helm_dd_interface_lines.  Pointers may be host or device, as for fields. */

/* L = 2(J-1); the padded columns of the interface lines (beta_j+1, beta_j+2 for
 * j = 1..J-1, in that order) are written to cols[0..min(L, cap)-1]. */
int helm_dd_interface_lines(const helm_dd* h, int* cols, int cap);

/* Algorithm 2 (Eq. reduce_compute_ut): u~^(j) solves A^(j) u~^(j) = f restricted
 * to D~^(j) = {beta_{j-1}+2 .. beta_j+1} (from column 0 for the first strip, to
 * N[0]-1 for the last), u~ = u~^(j) on D~^(j); phi = f - A u~, which vanishes
 * off the interface lines, is written in reduced form.  The J strip solves are
 * independent.  ut (a full field per right-hand side) may be NULL; phi may be
 * NULL when J = 1.  HELM_ESTATE before helm_dd_factor. */
helm_status helm_dd_reduce_rhs(helm_dd* h, const double* f, double* phi, double* ut, int nrhs);

/* Algorithm 3 on reduced arrays: out = R A P E in, with E the extension by zero
 * to the padded grid and R the restriction to the interface lines (the forward
 * sweep, the residual, the backward sweep and A applied to P E in; the result is
 * supported on the interface lines up to rounding).  in and out distinct. */
helm_status helm_dd_apply_AP_reduced(helm_dd* h, const double* in, double* out, int nrhs);

/* Algorithm 5 in the reduced space: phi from Algorithm 2, GMRES(restart) on
 * R A P E xi = phi (Eq. solve_A_reduced with psi = P E xi; vectors of N[2] N[1] L
 * entries per right-hand side, x0 = 0), u = P E xi + u~ (Algorithm 4).  GMRES
 * stops when the reduced residual would bring ||f - A u|| to tol ||f|| (in
 * mixed precision at 1e-3 of its right-hand side at the tightest: the complex64
 * operator is linear only up to its rounding); the true residual is then
 * formed on the whole grid in FP64 and, where it is still above tol ||f||
 * (complex64 strip solves leave small residuals off the lines, which the
 * reduced space does not see), the same steps are repeated on it (defect
 * correction, at most 8 passes).  info: GMRES iterations summed over the
 * passes, the true relative residual, the batch time.  Right-hand sides run in
 * panels (helm_dd_set_panel).  HELM_ENOTCONV (u and info written) when the
 * tolerance is not reached within maxit iterations. */
helm_status helm_dd_solve_reduced(helm_dd* h, const double* rhs, double* u, int nrhs, double tol, int restart,
                                  int maxit, helm_rhs_info* info);

/* Least-squares misfit J = 1/2 sum_s ||R u_s - d_s||^2 and its gradient with
 * respect to m = 1/c^2 on the interior grid (not in the paper: the adjoint of
 * A(m) = L - omega^2 diag(m)).  Sources are discrete deltas 1/h^dim at the
 * padded linear indices src_idx; R samples u at rec_idx; d is complex128
 * [nsrc][nrec] interleaved.  Forward and adjoint solves (A mu_s =
 * S^-1 conj(R^T r_s)) share the factors; grad = omega^2 Re sum_s S mu_s u_s,
 * folded from the padded grid onto the interior through the clamp extension.
 * The PML profile is held fixed.  misfit and grad_m (interior size) are
 * written; tol is the GMRES tolerance of both solves.  grad_m may be NULL:
 * then only the forward solves run and only the misfit is written.  Sources
 * are processed in panels (helm_dd_set_panel; by default as many as the free
 * device memory holds): a panel's forward fields are kept only until its
 * adjoint solves are done. */
helm_status helm_dd_gradient(helm_dd* h, const int64_t* src_idx, int nsrc,
                             const int64_t* rec_idx, int nrec, const double* d,
                             double tol, double* misfit, double* grad_m);

/* Order all device work of the handle on this cudaStream_t (NULL = the handle's
 * own stream).  The output passes of a sweep run on an internal low-priority
 * stream beside the strip solves; every call joins it back to this stream (an
 * event wait) before the call's results are used.  The caller keeps ownership
 * of the stream. */
helm_status helm_dd_set_stream(helm_dd* h, void* stream);

/* Per-kernel timing of the calls that follow: when enabled, each launch of the
 * library's kernels is bracketed by CUDA events on the launching stream and its
 * duration accumulated by kernel name.  helm_dd_kernel_stats copies up to cap
 * entries (name, launches, total ms) and returns how many exist. */
helm_status helm_dd_set_timing(helm_dd* h, int enable);
int helm_dd_kernel_stats(helm_dd* h, char (*names)[48], int64_t* launches,
                         double* total_ms, int cap);

/* Bytes of factor data one preconditioner application reads by the method's
 * own count (2 passes x sum over strip solves of N_y n_j^2 x element size, with
 * n_j = W_j in 2-D and W_j N_z in 3-D). */
double helm_dd_precond_factor_bytes(const helm_dd* h);

/* Padded sizes N[0..2]; strip widths W_j (J entries) when W != NULL. */
void helm_dd_dims(const helm_dd* h, int64_t N[3]);
int helm_dd_strip_widths(const helm_dd* h, int* W, int cap);
int helm_dd_interfaces(const helm_dd* h, int* beta, int cap);

void helm_dd_destroy(helm_dd* h);
const char* helm_dd_last_error(const helm_dd* h);

#ifdef __cplusplus
}
#endif
#endif /* HELM_DD_H */
