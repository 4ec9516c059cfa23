// Host-side declarations shared by the helm_dd translation units: the kernel
// timer and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "common.cuh"

namespace helm {

// Brackets launches with CUDA events on the launching stream and accumulates
// their durations per kernel name (only while enabled).
struct KernelTimer {
    bool enabled = false;
    struct Pending { int id; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<std::string> names;
    std::vector<int64_t> counts;
    std::vector<double> total_ms;
    std::vector<cudaEvent_t> pool;

    int id_of(const char* name) {
        for (size_t i = 0; i < names.size(); ++i)
            if (names[i] == name) return (int)i;
        names.emplace_back(name);
        counts.push_back(0);
        total_ms.push_back(0.0);
        return (int)names.size() - 1;
    }
    cudaEvent_t get_event() {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    // Resolve all pending pairs (call after the stream has been synchronised).
    void flush() {
        for (auto& p : pending) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
                counts[p.id] += 1;
                total_ms[p.id] += ms;
            }
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pending.clear();
    }
    void reset() { flush(); for (auto& c : counts) c = 0; for (auto& t : total_ms) t = 0; }
    ~KernelTimer() {
        for (auto& p : pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

struct TimedLaunch {
    KernelTimer* t;
    cudaStream_t s;
    int id = -1;
    cudaEvent_t a = nullptr;
    TimedLaunch(KernelTimer* tm, const char* name, cudaStream_t st) : t(tm), s(st) {
        if (t && t->enabled) {
            id = t->id_of(name);
            a = t->get_event();
            cudaEventRecord(a, s);
        }
    }
    ~TimedLaunch() {
        if (t && t->enabled && a) {
            cudaEvent_t b = t->get_event();
            cudaEventRecord(b, s);
            t->pending.push_back({id, a, b});
        }
    }
};

// ---- factor.cu
// shared memory of a factor kernel with nbuf W x W buffers (3, or 4 for the
// level-2 separator system)
constexpr size_t kFactorSmemMax = 227 * 1024;
size_t factor_smem_bytes(int Wmax, size_t esize, int nbuf);
// pool: Sinv, GT, GB (per grid row), Rinv, E, F, GT2, GB2, P2L, P2U (per separator)
template <typename C>
cudaError_t launch_factor(const Geom& g, int Wmax, void* const* pool, int* status, cudaStream_t s, KernelTimer* tm);

// ---- sweep.cu: one strip solve of the sweep.
// Right-hand side of strip st for row k, column c (padded column gc = lo-lpml+c):
//   r = [mlo <= gc <= mhi] src(b,k,gc) + [gc == t0 or gc == t0+1] tcoef * tin(b,k)
// solved for x on the strip grid; then x is scattered to dst on padded columns
// olo..ohi (dst = x, or dst = base + x when base != null) and the transfer
// difference tout(b,k) = x(to1) - x(to0) (strip-local columns) is written.
struct SweepStep {
    const double2* src;     // [B][Ny][Nx] FP64
    int mlo, mhi;           // mask of src columns entering the right-hand side
    int prev;               // strip whose solve passes its transfer into this one, or -1
    int pdir;               // that strip's transfer columns: 0 forward (its right end), 1 backward (its left end)
    int t0;                 // first padded column receiving the transfer
    double tcoef;           // transfer coefficient (-1/h^2 forward, +1/h^2 backward)
    // Robin transmission (Section 4.4): the transfer is tcoef (rbk[k] x_in + x_out) with
    // x_in = x(to[rb_in]) (the receiving strip's boundary column) and x_out the other
    // transfer column; null for the PML transfer tcoef (x(to1) - x(to0))
    const double2* rbk;
    int rb_in;
};

// Separator-parts buffer of one strip solve for B right-hand sides (sweep.cu): the parts,
// then every chunk's contributions to the level-2 right-hand sides.
size_t sweep_parts_bytes(int P, int B, int Wmax, size_t esize);
size_t sweep_parts_total_bytes(int P, int B, int Wmax, size_t esize);
size_t sweep_parts2_bytes(int P, int B, int Wmax, size_t esize);   // the trailing level-2 accumulators
struct SweepWork {
    void* ybuf;             // [B][Ny][Wmax] working precision (this strip's chain solution)
    void* parts;            // sweep_parts_total_bytes: parts, then level-2 contributions
    int* counters;          // [RHS tile][G+1], zero between launches
    int* status;            // error word (7 = bounded wait timed out)
    int Wmax;               // row stride of ybuf and parts: even, >= every strip width
    int B;
    int zrows;              // longest chain of one CTA (chunk rows, group size, G-1)
    const void* pybuf;      // the previous strip solve's chain solution (when SweepStep::prev >= 0)
    // launch with programmatic stream serialisation (the next strip solve's CTAs stage their
    // blocks while this one finishes); off where strip solves of several streams share the SMs
    bool pdl = true;
};

// Output pass of a sweep (k_sweep_output) over strips jlo .. jlo+nstrip-1,
// after their strip solves.
struct OutArgs {
    Geom g;
    int dir;                // output ranges of the forward (0) or backward (1) sweep
    int jlo, nstrip;
    const void* ybuf;       // strip j's chain solution at ybuf + j*ystride (elements)
    int64_t ystride;
    int Wmax, B, Bt;
    double2* dst;           // [B][Ny][Nx] output field
    const double2* base;    // optional field added on output
    int maxcta;             // CTAs of the launch (0: one per work item)
};
template <typename C>
cudaError_t launch_outputs(const OutArgs& O, void* const* pool, cudaStream_t s, KernelTimer* tm);

// Whether one strip solve of st (a ring of at least four W x W blocks in shared memory)
// fits on an SM with elements of esize bytes.
bool strip_solve_fits(const StripDev& st, int zrows, size_t esize);

template <typename C>
// pst: the strip of the previous solve whose transfer enters this one (step.prev >= 0), host copy
cudaError_t launch_strip_solve(const Geom& g, int j, const StripDev& st_host, const StripDev* pst,
                               const SweepStep& step, const SweepWork& wk, void* const* pool, cudaStream_t s,
                               KernelTimer* tm);

// ---- slab3d.cu: strips of a 3-D grid (one dense block of n = W N_z unknowns per row y)
// Scratch of the factorisation: the block being inverted (column-major, ldm >= n),
// the published exchanged pivot columns (n x ldm, one per elimination step), the row
// exchanges and their inverse, the published pivot rows (n) and the step counter.
struct SlabScratch {
    void* M;
    void* mult;
    int ldm;
    int* perm;
    int* pinv;
    int* pivrow;
    unsigned* bar;
};
// One strip solve: right-hand sides and solution [B][Ny][ld], the previous strip
// solve's solution (for the transfer), s_x s_z per block entry, s_z in the table ct.
struct SlabWork {
    void* rbuf;
    void* ybuf;
    const void* pybuf;
    const void* sxz;          // this strip's s_x(c) s_z(z), working precision, n entries
    int64_t ct_sz;            // offset of s_z(z) in Geom::ct
    const double2* cy_host;   // host: -alpha_y(y_{k-1/2}) / h^2, k = 0 .. Ny
    int ld;                   // row stride of rbuf / ybuf / pybuf (>= every strip's n)
    int B;
    unsigned* bar;            // grid-barrier counter of the strip-solve kernel
    int* status;              // error word (7 = a bounded wait gave up)
};
// Factor blocks X_k = S_k^{-1} of strip st into pool + st.fac (row-major, leading
// dimension st.ld, st.bs elements per block), k = 0 .. Ny-1.
template <typename C>
cudaError_t launch_slab_factor(const Geom& g, const StripDev& st, void* pool, const SlabScratch& sc, int* status,
                               cudaStream_t s, KernelTimer* tm);
// M (column-major, leading dimension ldm) = D_k - C_k Xp C_k (Xp = X_{k-1} in the sweep
// layout, leading dimension ld; M = D_k when Xp is null).
template <typename C>
cudaError_t launch_slab_build(const Geom& g, const StripDev& st, int k, const C* Xp, int ld, C* M, int ldm,
                              cudaStream_t s, KernelTimer* tm);
// slab_tc.cu: the blocks X_k = S_k^{-1}, k = 0 .. Ny-1, of up to 8 strips side by side in
// complex64, inverted by blocked Gauss-Jordan elimination whose rank-12 updates run on the
// tensor cores; scratch of slab_factor_tc_scratch(max n, strips) bytes.
size_t slab_factor_tc_scratch(int nmax, int ns);
cudaError_t launch_slab_factor_tc(const Geom& g, const StripDev* strips, int ns, void* pool, void* scratch,
                                  int* status, cudaStream_t s, KernelTimer* tm);
// Right-hand side and block forward / back substitution of strip st (into wk.ybuf).
template <typename C>
cudaError_t launch_slab_solve(const Geom& g, const StripDev& st, const StripDev* pst, const SweepStep& sp,
                              const SlabWork& wk, const void* pool, cudaStream_t s, KernelTimer* tm);
// dst = [base +] the strip solution on padded columns st.olo[dir] .. st.ohi[dir].
template <typename C>
cudaError_t launch_slab_out(const Geom& g, const StripDev& st, int dir, const void* ybuf, int ld, double2* dst,
                            const double2* base, int B, cudaStream_t s, KernelTimer* tm);

// Load the modules of each file's kernels onto the current device (lazy module
// loading would otherwise load them, and take their memory, at the first launch
// inside some later call).
cudaError_t preload_sweep_kernels();
cudaError_t preload_slab_kernels();
cudaError_t preload_field_kernels();

// ---- field.cu: FP64 grid kernels
cudaError_t launch_k2(const double* c_int, double* k2, int dim, int nx, int ny, int nz, int w, double omega,
                      cudaStream_t s);
// out = (f ? f - A u : A u), paper form, B fields
cudaError_t launch_stencil(const Geom& g, const double2* u, const double2* f, double2* out, int B,
                           cudaStream_t s, KernelTimer* tm);
cudaError_t launch_copy_cols(const double2* src, double2* dst, int B, int Nx, int Ny, int Nz, int xlo, int xhi,
                             cudaStream_t s, KernelTimer* tm);
// partial[b][i][blk] for h[b][i] = sum_n conj(V_i[b][n]) w[b][n]; V_i at V + i*vstride
cudaError_t launch_multidot(const double2* V, int64_t vstride, const double2* w, int nv, int B, int64_t N,
                            double2* partial, int nblk, double2* out, cudaStream_t s, KernelTimer* tm);
// w[b] += sum_i coef[b][i] V_i[b]  (coef device [B][nv])
cudaError_t launch_multi_axpy(double2* w, const double2* V, int64_t vstride, const double2* coef, int nv,
                              int B, int64_t N, cudaStream_t s, KernelTimer* tm);
// dst[b] = src[b] * scale[b] (scale real, device [B])
cudaError_t launch_scale(double2* dst, const double2* src, const double* scale, int B, int64_t N,
                         cudaStream_t s, KernelTimer* tm);
// gpad += omega^2 Re sum_s S mu_s u_s
cudaError_t launch_grad_accum(const double2* U, const double2* MU, const Geom& g, int nsrc, double* gpad,
                              cudaStream_t s);
cudaError_t launch_fold(const double* gpad, double* gint, int dim, int nx, int ny, int nz, int w, cudaStream_t s);
cudaError_t launch_gather(const double2* U, int64_t ustride, const int64_t* idx, int nidx, int B,
                          double2* out, cudaStream_t s);
// Interface lines of the reduced space (Section 2.3): red[r * L + i] = column cols[i] of
// grid row r, rows r = 0 .. B N_z N_y - 1.
cudaError_t launch_gather_cols(const double2* full, double2* red, const int* cols, int L, int64_t rows, int Nx,
                               cudaStream_t s, KernelTimer* tm);
cudaError_t launch_scatter_cols(const double2* red, double2* full, const int* cols, int L, int64_t rows, int Nx,
                                cudaStream_t s, KernelTimer* tm);
// out (reduced) = f - A u on the interface columns, f from the full field f_full or the
// reduced f_red (out = A u there when both are null)
cudaError_t launch_stencil_cols(const Geom& g, const double2* u, const double2* f_full, const double2* f_red,
                                double2* out, const int* cols, int L, int B, cudaStream_t s, KernelTimer* tm);
// dst += src (n complex entries)
cudaError_t launch_add(double2* dst, const double2* src, int64_t n, cudaStream_t s, KernelTimer* tm);
// dst[b * stride + idx[b*n + i]] = val[b*n + i]  (device idx / val, B fields of n points)
cudaError_t launch_scatter(double2* dst, int64_t stride, const int64_t* idx, const double2* val, int n, int B,
                           cudaStream_t s);

}  // namespace helm
