// Three-dimensional strips (Section 2.2, Algorithm 1 and the sweeps of Section
// 2.1 on a 3-D grid).  A strip is a slab of W x-columns by all N_z planes; at
// grid row y = k its unknowns form one block of n = W N_z points, ordered
// e = z W + c (strip-local column c fastest).  S^(j) A^(j) is block tridiagonal
// along y with these dense-after-elimination blocks and diagonal couplings:
//   D_k(e,e)     = [s_y s_z (a_x(c+1/2) + a_x(c-1/2))
//                   + s_x s_z (a_y(k+1/2) + a_y(k-1/2))
//                   + s_x s_y (a_z(z+1/2) + a_z(z-1/2))] / h^2 - s_x s_y s_z k^2
//   D_k(e,e+1)   = -s_y s_z a_x(c+1/2) / h^2            (c+1 < W, same plane)
//   D_k(e,e+W)   = -s_x s_y a_z(z+1/2) / h^2
//   C_k(e)       = -s_x(c) s_z(z) a_y(k-1/2) / h^2      (couples rows k-1, k)
// with s = 1/alpha at integer points and a = alpha at half points.
//
// Factorisation (Algorithm 1, top down): X_k = S_k^{-1},
//   S_0 = D_0,  S_k = D_k - C_k X_{k-1} C_k,
// each S_k inverted by Gauss-Jordan elimination with partial (row) pivoting on
// the whole GPU (one cooperative launch per block).  Solve of a strip
// (block forward and back substitution):
//   y_k = X_k (r_k - C_k y_{k-1}),   k = 0 .. N_y-1
//   x_k = y_k - X_k C_{k+1} x_{k+1}, k = N_y-2 .. 0
// all 2 N_y - 1 steps in one cooperative launch (k_slab_sweep), each a
// matrix-vector product that streams X_k from HBM through shared memory.
#include <algorithm>

#include <type_traits>

#include "common.cuh"
#include "strip_ops.cuh"
#include "internal.h"

namespace helm {
namespace {

constexpr uint32_t kBarPolls = 1u << 20;   // polls of a grid barrier before it gives up (about a second)
constexpr int kGjThreads = 256;
constexpr int kGjRowsPerThread = 8;        // n <= kGjThreads * kGjRowsPerThread
constexpr int kGjMaxCols = 64;             // columns owned by one CTA

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <typename C> __device__ __forceinline__ C ldcg(const C* p);
template <> __device__ __forceinline__ float2 ldcg(const float2* p) { return __ldcg(p); }
template <> __device__ __forceinline__ double2 ldcg(const double2* p) { return __ldcg(p); }

// One thread waits (bounded) until the counter reaches target; a wait that gives up
// records 7 in the status word and returns false.
__device__ bool wait_count(const unsigned* ctr, unsigned target, int* status) {
    unsigned v = ld_acquire_gpu(ctr);
    for (uint32_t it = 0; v < target && it < kBarPolls; ++it) {
        __nanosleep(20);
        v = ld_acquire_gpu(ctr);
    }
    if (v >= target) return true;
    atomicExch(status, 7);
    return false;
}
__device__ __forceinline__ void add_release(unsigned* ctr) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ctr) : "memory");
}

// ------------------------------------------------------------ block entries
__device__ __forceinline__ double2 slab_sz(const Geom& g, int z) { return cinv(g.gz_int[z]); }

__device__ double2 slab_diag(const Geom& g, const StripDev& st, int k, int c, int z) {
    const double2 sx = strip_sx(g, st, c), sy = glob_sy(g, k), sz = slab_sz(g, z);
    const double2 xs = cadd(strip_ax_half(g, st, c + 1), strip_ax_half(g, st, c));
    const double2 ys = cadd(g.gy_half[k + 1], g.gy_half[k]);
    const double2 zs = cadd(g.gz_half[z + 1], g.gz_half[z]);
    double2 d = cadd(cadd(cmul(cmul(sy, sz), xs), cmul(cmul(sx, sz), ys)), cmul(cmul(sx, sy), zs));
    d = cscale(d, g.inv_h2);
    const double k2 = g.k2[((int64_t)z * g.Ny + k) * g.Nx + strip_k2_col(st, c)];
    return csub(d, cscale(cmul(cmul(sx, sy), sz), k2));
}
// entry (e, e+1), e = z W + c, c + 1 < W
__device__ double2 slab_xoff(const Geom& g, const StripDev& st, int k, int c, int z) {
    return cscale(cmul(cmul(glob_sy(g, k), slab_sz(g, z)), strip_ax_half(g, st, c + 1)), -g.inv_h2);
}
// entry (e, e+W), z + 1 < N_z
__device__ double2 slab_zoff(const Geom& g, const StripDev& st, int k, int c, int z) {
    return cscale(cmul(cmul(strip_sx(g, st, c), glob_sy(g, k)), g.gz_half[z + 1]), -g.inv_h2);
}
// D_k(r, a) for any pair (zero off the stencil)
__device__ double2 slab_dentry(const Geom& g, const StripDev& st, int k, int r, int a) {
    const int W = st.W;
    const int lo = imin(r, a), d = r > a ? r - a : a - r;
    if (d != 0 && d != 1 && d != W) return make_double2(0.0, 0.0);
    const int c = lo % W, z = lo / W;
    if (d == 0) return slab_diag(g, st, k, c, z);
    if (d == 1 && c + 1 < W) return slab_xoff(g, st, k, c, z);
    if (d == W) return slab_zoff(g, st, k, c, z);
    return make_double2(0.0, 0.0);
}

// M (column-major, ldm) = - C_k Xp C_k, Xp = X_{k-1} in the row-major sweep layout
// (leading dimension ld), or M = 0 for k = 0; k_slab_dadd then adds D_k.  32 x 32 tiles.
template <typename C>
__global__ void __launch_bounds__(256) k_slab_build(Geom g, StripDev st, int k, const C* __restrict__ Xp, int ld,
                                                    C* __restrict__ M, int ldm) {
    __shared__ C tile[32][33];
    __shared__ C cr[32], cc[32];
    const int n = st.W * g.Nz;
    const int r0 = blockIdx.y * 32, a0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 8 rows of 32
    if (Xp) {
        for (int i = ty; i < 32; i += 8) {
            const int r = r0 + i, a = a0 + tx;
            tile[i][tx] = (r < n && a < n) ? Xp[(int64_t)r * ld + a] : CT<C>::zero();
        }
        if (threadIdx.x < 64) {
            const int e = (threadIdx.x < 32 ? r0 : a0) + tx;
            // C_k(e) = s_x(c) s_z(z) (-alpha_y(y_{k-1/2}) / h^2) from the working-precision table
            const C* ct = reinterpret_cast<const C*>(g.ct);
            const C v = e < n ? cmul(cmul(ct[st.ctab + e % st.W], ct[g.ct_sz + e / st.W]), ct[g.ct_cy + k])
                              : CT<C>::zero();
            (threadIdx.x < 32 ? cr : cc)[tx] = v;
        }
    }
    __syncthreads();
    // write column a0+i, rows r0+tx (coalesced along rows)
    for (int i = ty; i < 32; i += 8) {
        const int a = a0 + i, r = r0 + tx;
        if (a >= n || r >= n) continue;
        M[(int64_t)a * ldm + r] = Xp ? cneg(cmul(cmul(cr[tx], tile[tx][i]), cc[i])) : CT<C>::zero();
    }
}

// M(r, a) += D_k(r, a) on the stencil entries of row r: a = r, r +- 1 (same z), r +- W; one
// entry per thread (the entries are evaluated in FP64, so they are spread over the GPU).
template <typename C>
__global__ void __launch_bounds__(64) k_slab_dadd(Geom g, StripDev st, int k, C* __restrict__ M, int ldm) {
    const int n = st.W * g.Nz, W = st.W;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 5 * n; e += gridDim.x * blockDim.x) {
        const int r = e / 5, i = e % 5, c = r % W;
        const int a = i == 0 ? r : i == 1 ? (c > 0 ? r - 1 : -1) : i == 2 ? (c + 1 < W ? r + 1 : -1) : i == 3 ? r - W : r + W;
        if (a < 0 || a >= n) continue;
        C* p = M + (int64_t)a * ldm + r;
        *p = cadd(*p, CT<C>::from(slab_dentry(g, st, k, r, a)));
    }
}

// In-place Gauss-Jordan inverse with partial pivoting of the n x n matrix M
// (column-major, ldm), columns dealt round-robin to the CTAs of a cooperative
// launch.  Step i: rows i and p (the largest |M(r,i)|, r >= i) are exchanged,
// the pivot row is scaled by 1/M(p,i) with M(i,i) <- 1/pivot, and every other
// row r loses m_r times it with M(r,i) <- -m_r/pivot (m_r = M(r,i) after the
// exchange).  The owner of column i publishes p and the exchanged column m (one
// buffer per step, never reused, so a CTA may trail the others by any number of
// steps) and raises the published-step counter bar[0] (release, zero at launch); a
// CTA starts step i once that counter says so (acquire).  Only the owner of the next
// column, which it updates first, is on the critical path.  The
// result is (P M)^{-1} for the product P of the exchanges; pinv[c] = the
// position of original row c after all exchanges, so M^{-1}(:, c) = result(:, pinv[c]).
// cached != 0: a CTA keeps its columns in shared memory for the whole elimination.
template <typename C>
__global__ void __launch_bounds__(kGjThreads) k_gj_invert(C* __restrict__ M, int n, int ldm, int* __restrict__ perm,
                                                         int* __restrict__ pinv, C* __restrict__ mult,
                                                         int* __restrict__ pivrow, unsigned* __restrict__ bar,
                                                         int* __restrict__ status, int cached) {
    using R = typename CT<C>::R;
    extern __shared__ __align__(16) unsigned char gj_smem[];
    __shared__ C s_ai[kGjMaxCols], s_ap[kGjMaxCols];
    __shared__ R s_best[kGjThreads / 32];
    __shared__ int s_bidx[kGjThreads / 32];
    __shared__ int s_p, s_ok;
    __shared__ int s_rows[kGjThreads * kGjRowsPerThread];
    const int nb = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
    const int ncol = b < n ? (n - 1 - b) / nb + 1 : 0;   // owned columns b, b+nb, ...
    C* cache = reinterpret_cast<C*>(gj_smem);            // [ncol][n] when cached
    auto colp = [&](int lc) -> C* {
        return cached ? cache + (int64_t)lc * n : M + (int64_t)(b + lc * nb) * ldm;
    };
    if (cached) {
        for (int lc = 0; lc < ncol; ++lc)
            for (int r = tid; r < n; r += kGjThreads) cache[(int64_t)lc * n + r] = M[(int64_t)(b + lc * nb) * ldm + r];
        __syncthreads();
    }

    // pivot search and publication for column i (owned by this CTA, up to date)
    auto publish = [&](int i) {
        const C* col = colp(i / nb);   // i = b + (i / nb) nb
        R best = (R)-1;
        int bi = n;
        for (int r = i + tid; r < n; r += kGjThreads) {
            const R v = cabs2(col[r]);
            if (v > best) { best = v; bi = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const R ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if ((tid & 31) == 0) { s_best[tid >> 5] = best; s_bidx[tid >> 5] = bi; }
        __syncthreads();
        if (tid == 0) {
            R bb = s_best[0];
            int bx = s_bidx[0];
            for (int w = 1; w < kGjThreads / 32; ++w)
                if (s_best[w] > bb || (s_best[w] == bb && s_bidx[w] < bx)) { bb = s_best[w]; bx = s_bidx[w]; }
            if (!(bb > (R)0) || !(bb < (R)INFINITY) || bx >= n) {
                atomicExch(status, 6);   // zero or non-finite pivot: the result is invalid
                bx = i;
            }
            s_p = bx;
            pivrow[i] = bx;
        }
        __syncthreads();
        const int p = s_p;
        C* mu = mult + (int64_t)i * ldm;
        for (int r = tid; r < n; r += kGjThreads) mu[r] = col[r == i ? p : (r == p ? i : r)];
        __syncthreads();
        if (tid == 0) add_release(bar);   // step i published
    };

    if (b == 0 && ncol > 0) publish(0);   // column 0 belongs to CTA 0
    for (int i = 0; i < n; ++i) {
        if (tid == 0) s_ok = wait_count(bar, (unsigned)(i + 1), status);
        __syncthreads();
        if (!s_ok) return;
        const int p = __ldcg(pivrow + i);
        const C* mu = mult + (int64_t)i * ldm;
        const C ip = cinv(ldcg(mu + i));
        if (b == 0 && tid == 0) perm[i] = p;
        C m_r[kGjRowsPerThread];
#pragma unroll
        for (int u = 0; u < kGjRowsPerThread; ++u) {
            const int r = tid + u * kGjThreads;
            m_r[u] = r < n ? ldcg(mu + r) : CT<C>::zero();
        }
        for (int lc = tid; lc < ncol; lc += kGjThreads) {
            const C* col = colp(lc);
            s_ai[lc] = col[i];
            s_ap[lc] = col[p];
        }
        __syncthreads();
        auto update = [&](int lc) {
            const int c = b + lc * nb;
            C* col = colp(lc);
            const C t = c == i ? ip : cmul(s_ap[lc], ip);
            const C ai = s_ai[lc];
#pragma unroll
            for (int u = 0; u < kGjRowsPerThread; ++u) {
                const int r = tid + u * kGjThreads;
                if (r >= n) continue;
                const C base = c == i ? CT<C>::zero() : (r == p ? ai : col[r]);
                col[r] = r == i ? t : csub(base, cmul(m_r[u], t));
            }
        };
        const int cn = i + 1;
        const int lcn = (cn < n && cn % nb == b) ? cn / nb : -1;
        if (lcn >= 0) {
            update(lcn);
            __syncthreads();
            publish(cn);
        }
        for (int lc = 0; lc < ncol; ++lc)
            if (lc != lcn) update(lc);
        __syncthreads();   // s_ai / s_ap are rewritten at the next step
    }
    if (cached) {
        __syncthreads();
        for (int lc = 0; lc < ncol; ++lc)
            for (int r = tid; r < n; r += kGjThreads) M[(int64_t)(b + lc * nb) * ldm + r] = cache[(int64_t)lc * n + r];
    }
    // the exchanges, replayed: s_rows[r] = original row at position r
    if (b == 0) {
        __syncthreads();
        for (int r = tid; r < n; r += kGjThreads) s_rows[r] = r;
        __syncthreads();
        if (tid == 0)
            for (int i = 0; i < n; ++i) {
                const int p = perm[i], t = s_rows[i];
                s_rows[i] = s_rows[p];
                s_rows[p] = t;
            }
        __syncthreads();
        for (int r = tid; r < n; r += kGjThreads) pinv[s_rows[r]] = r;
    }
}

// X (row-major sweep layout, ld, columns n..ld-1 zero) = M^{-1} from the
// Gauss-Jordan result: X(a, c) = Mgj(a, pinv[c]) = M[pinv[c] * ldm + a].
template <typename C>
__global__ void __launch_bounds__(256) k_slab_store(const C* __restrict__ M, int n, int ldm,
                                                    const int* __restrict__ pinv, C* __restrict__ X, int ld) {
    __shared__ C tile[32][33];
    const int a0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int i = ty; i < 32; i += 8) {   // column c0+i of X: rows a0+tx (contiguous in M)
        const int c = c0 + i, a = a0 + tx;
        tile[i][tx] = (c < n && a < n) ? M[(int64_t)pinv[c] * ldm + a] : CT<C>::zero();
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const int a = a0 + i, c = c0 + tx;
        if (a < n && c < ld) X[(int64_t)a * ld + c] = tile[tx][i];
    }
}

// ------------------------------------------------------------------ sweeps
// Right-hand side of a strip solve in the symmetric form (as the 2-D sweep):
//   r(b,k,e) = s_x s_y s_z ([mlo <= gc <= mhi] src(b,z,k,gc)
//                           + [gc == t0 or t0+1] tcoef (xp(to1) - xp(to0)))
// xp: the previous strip solve's solution (strip pst, its transfer columns).
template <typename C>
__global__ void k_slab_rhs(Geom g, StripDev st, SweepStep sp, StripDev pst, const C* __restrict__ ct,
                           int64_t ct_sz, const C* __restrict__ prevY, int pld, C* __restrict__ Rb, int ld, int B) {
    const int W = st.W, Nz = g.Nz, Ny = g.Ny, n = W * Nz;
    const int cofs = st.lo - st.lpml;
    const int64_t tot = (int64_t)B * Ny * ld;
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < tot; o += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(o % ld);
        const int k = (int)((o / ld) % Ny);
        const int b = (int)(o / ((int64_t)ld * Ny));
        if (e >= n) { Rb[o] = CT<C>::zero(); continue; }
        const int c = e % W, z = e / W, gc = cofs + c;
        const C s = cmul(cmul(ct[st.ctab + c], ct[g.ct_sy + k]), ct[ct_sz + z]);
        double2 f = make_double2(0.0, 0.0);
        if (gc >= sp.mlo && gc <= sp.mhi) f = sp.src[(((int64_t)b * Nz + z) * Ny + k) * g.Nx + gc];
        C v = cmul(CT<C>::from(f), s);
        if (prevY && (gc == sp.t0 || gc == sp.t0 + 1)) {
            const C* py = prevY + ((int64_t)b * Ny + k) * pld + (int64_t)z * pst.W;
            const C tv = csub(py[pst.xc[2 * sp.pdir + 1]], py[pst.xc[2 * sp.pdir]]);
            v = cadd(v, cmul(cscale(tv, (typename CT<C>::R)sp.tcoef), s));
        }
        Rb[o] = v;
    }
}

// A whole strip solve (2 N_y - 1 block steps) in one cooperative launch of at most
// one CTA per SM.  CTA b owns rows [b rpc, (b+1) rpc) of every block; step s is
//   forward  (s < N_y):      y_k = X_k (r_k - C_k y_{k-1}),       k = s
//   backward (s >= N_y):     x_k = y_k - X_k (C_{k+1} x_{k+1}),    k = 2 N_y - 2 - s
// in place in Y.  A producer warp streams the CTA's rows of X_k, step after step,
// into a ring of row slots in shared memory (cp.async.bulk + mbarriers), with the
// next step's rows prefetched into L2; it never waits for the vector, so the factor
// stream runs ahead across the steps while the compute warps wait at the grid barrier
// for the previous step's rows.  Compute warp w owns the column segment
// [w seg, (w+1) seg) of every row: it loads its part of the step's input vector
// z = r_k - C y_kp straight into registers, forms its partial products for all rows
// of the step (four rows at a time), and the eight partials of a row are summed in
// shared memory.  Every wait is bounded: on time-out the kernel records 7 in the
// status word, waits (bounded) for its copies in flight and returns.
template <typename C>
struct SlabSweepArgs {
    const C* X;          // block 0 of the strip; block k at X + k * bs, row-major, leading dimension xld
    int64_t bs;
    int n, xld, Ny, rpc, ring;
    const C* rhs;        // [B][Ny][ld] right-hand sides
    C* Y;                // [B][Ny][ld] solution
    int ld, B;           // row stride of rhs / Y; right-hand sides of this launch (<= NB)
    const C* sxz;        // s_x(c) s_z(z) per block entry
    const C* cyt;        // -alpha_y(y_{k-1/2}) / h^2, k = 0 .. Ny
    unsigned* bar;       // step counter, zero at launch
    int* status;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mb_init(uint64_t* m, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_expect_tx(uint64_t* m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mb_arrive(uint64_t* m) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(m)) : "memory");
}
__device__ __forceinline__ bool mb_wait(uint64_t* m, uint32_t parity) {
    for (uint32_t it = 0; it < kBarPolls; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_addr(m)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void bulk_row(void* dst, const void* src, uint32_t bytes, uint64_t* m) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(m))
        : "memory");
}
__device__ __forceinline__ void compute_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

constexpr int kSweepThreads = 288;   // 8 compute warps + 1 producer warp
constexpr int kMaxRpc = 32;          // rows per CTA and step

// kSegU: columns per lane, 8 warps x 32 lanes x kSegU >= xld (8: n <= 2048, 16: n <= 4096)
template <typename C, int NB, int kSegU>
__global__ void __launch_bounds__(kSweepThreads, 1) k_slab_sweep(SlabSweepArgs<C> A) {
    using R = typename CT<C>::R;
    extern __shared__ __align__(128) unsigned char sweep_smem[];
    const int R_ = A.ring, xld = A.xld;
    C* ring = reinterpret_cast<C*>(sweep_smem);                       // [ring][xld]
    C* part = ring + (int64_t)R_ * xld;                               // [8][kMaxRpc][NB] partial products
    uint64_t* full = reinterpret_cast<uint64_t*>(part + 8 * kMaxRpc * NB);   // [ring]
    uint64_t* empty = full + R_;                                      // [ring]
    int* abort_flag = reinterpret_cast<int*>(empty + R_);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r0 = blockIdx.x * A.rpc, nrow = imin(A.rpc, A.n - r0);
    const int nsteps = 2 * A.Ny - 1;
    const uint32_t rowbytes = (uint32_t)(xld * sizeof(C));
    // ring slots go back to the producer at the end of a step (after the grid arrival) when
    // the ring holds a whole step; otherwise each warp frees a group's slots as soon as it
    // has used them
    constexpr int RG = NB == 1 ? 4 : 2;
    const bool defer = R_ >= A.rpc;
    if (tid == 0) {
        for (int i = 0; i < R_; ++i) { mb_init(&full[i], 1); mb_init(&empty[i], defer ? 1 : 8); }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == 8) {   // producer
        if (lane == 0) {
            uint32_t g = 0;
            bool ok = true;
            // the CTA's rows of block k(s) into L2, one step ahead of the ring copies: the
            // ring holds about one step, the HBM stream then runs on across the barrier
            auto prefetch = [&](int s) {
                if (s >= nsteps) return;
                const int k = s < A.Ny ? s : 2 * A.Ny - 2 - s;
                const char* src = reinterpret_cast<const char*>(A.X + (int64_t)k * A.bs + (int64_t)r0 * xld);
                const uint32_t bytes = (uint32_t)nrow * rowbytes;
                for (uint32_t o = 0; o < bytes; o += 65536)
                    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src + o),
                                 "r"(bytes - o < 65536 ? bytes - o : 65536)
                                 : "memory");
            };
            prefetch(0);
            for (int s = 0; s < nsteps && ok; ++s) {
                prefetch(s + 1);
                const int k = s < A.Ny ? s : 2 * A.Ny - 2 - s;
                const C* src = A.X + (int64_t)k * A.bs + (int64_t)r0 * xld;
                for (int i = 0; i < nrow; ++i, ++g) {
                    const int slot = (int)(g % (uint32_t)R_);
                    const uint32_t use = g / (uint32_t)R_;
                    if (use > 0 && !mb_wait(&empty[slot], (use - 1) & 1)) { ok = false; break; }
                    if (*(volatile int*)abort_flag) { ok = false; break; }
                    mb_expect_tx(&full[slot], rowbytes);
                    bulk_row(ring + (int64_t)slot * xld, src + (int64_t)i * xld, rowbytes, &full[slot]);
                }
            }
            if (!ok) atomicExch(A.status, 7);
            // copies still in flight land before the CTA exits
            const uint32_t lo = g > (uint32_t)R_ ? g - (uint32_t)R_ : 0;
            for (uint32_t q = lo; q < g; ++q) mb_wait(&full[q % (uint32_t)R_], (q / (uint32_t)R_) & 1);
        }
        return;
    }

    // compute warps
    const int e0 = warp * 32 * kSegU + lane;   // this lane's columns: e0 + 32 u, u < kSegU
    uint32_t g0 = 0;   // issue index of this step's first row
    for (int s = 0; s < nsteps; ++s, g0 += (uint32_t)nrow) {
        const bool fwd = s < A.Ny;
        const int k = fwd ? s : 2 * A.Ny - 2 - s;
        const int kp = fwd ? k - 1 : k + 1;   // neighbouring row whose solution enters
        if (s > 0) {   // every CTA's rows of the previous step are written
            if (tid == 0) {
                const unsigned target = (unsigned)s * gridDim.x;
                unsigned v = ld_acquire_gpu(A.bar);
                for (uint32_t it = 0; v < target && it < kBarPolls; ++it) {
                    __nanosleep(20);
                    v = ld_acquire_gpu(A.bar);
                }
                if (v < target) { atomicExch(A.status, 7); *(volatile int*)abort_flag = 1; }
            }
            compute_sync();
            if (*(volatile int*)abort_flag) return;
        }
        // backward: y_k of the rows this CTA outputs (thread t < nrow B: row t / B, rhs t % B)
        const int ob = tid % NB, oi = tid / NB;
        const bool outs = tid < nrow * NB && ob < A.B;
        C* yo = A.Y + ((int64_t)imin(ob, A.B - 1) * A.Ny + k) * A.ld + r0 + imin(oi, nrow - 1);
        const C ybase = (outs && !fwd) ? *yo : CT<C>::zero();
        // z = r_k - cy sxz .* y_kp on this lane's columns, in registers
        const C cy = A.cyt[fwd ? k : k + 1];
        C z[kSegU][NB];
#pragma unroll
        for (int u = 0; u < kSegU; ++u) {
            const int e = e0 + 32 * u;
            const bool ok = e < A.n;
            const int ec = imin(e, A.n - 1);
            const C sc = cmul(cy, ok ? A.sxz[ec] : CT<C>::zero());
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const bool okb = ok && b < A.B;
                const int64_t rb = (int64_t)imin(b, A.B - 1) * A.Ny;
                const C r = (okb && fwd) ? ldcg(A.rhs + (rb + k) * A.ld + ec) : CT<C>::zero();
                const C y = (okb && kp >= 0) ? ldcg(A.Y + (rb + kp) * A.ld + ec) : CT<C>::zero();
                z[u][b] = csub(r, cmul(sc, y));
            }
        }
        // partial products of this warp's segment, RG rows at a time: the group's rows
        // are awaited first, then their products interleaved (independent chains)
        bool ok = true;
        for (int i0 = 0; i0 < nrow && ok; i0 += RG) {
            bool landed = true;
#pragma unroll
            for (int r = 0; r < RG; ++r) {
                const uint32_t g = g0 + (uint32_t)(i0 + r);
                if (i0 + r < nrow) landed &= mb_wait(&full[g % (uint32_t)R_], (g / (uint32_t)R_) & 1);
            }
            if (!__all_sync(0xffffffffu, landed)) { ok = false; break; }
            const C* xr[RG];
#pragma unroll
            for (int r = 0; r < RG; ++r)
                xr[r] = ring + (int64_t)((g0 + (uint32_t)imin(i0 + r, nrow - 1)) % (uint32_t)R_) * xld;
            C acc[RG][NB];
#pragma unroll
            for (int r = 0; r < RG; ++r)
#pragma unroll
                for (int b = 0; b < NB; ++b) acc[r][b] = CT<C>::zero();
#pragma unroll
            for (int u = 0; u < kSegU; ++u) {
                const int e = e0 + 32 * u;
                C x[RG];
#pragma unroll
                for (int r = 0; r < RG; ++r) x[r] = e < xld ? xr[r][e] : CT<C>::zero();
#pragma unroll
                for (int r = 0; r < RG; ++r)
#pragma unroll
                    for (int b = 0; b < NB; ++b) acc[r][b] = cfma(x[r], z[u][b], acc[r][b]);
            }
            if (!defer) {
                __syncwarp();
                if (lane == 0)
                    for (int r = 0; r < RG && i0 + r < nrow; ++r)
                        mb_arrive(&empty[(g0 + (uint32_t)(i0 + r)) % (uint32_t)R_]);
            }
#pragma unroll
            for (int r = 0; r < RG; ++r)
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    R re = acc[r][b].x, im = acc[r][b].y;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        re += __shfl_xor_sync(0xffffffffu, re, o);
                        im += __shfl_xor_sync(0xffffffffu, im, o);
                    }
                    acc[r][b].x = re;
                    acc[r][b].y = im;
                }
            if (lane == 0)
#pragma unroll
                for (int r = 0; r < RG; ++r)
                    if (i0 + r < nrow)
#pragma unroll
                        for (int b = 0; b < NB; ++b) part[(warp * kMaxRpc + i0 + r) * NB + b] = acc[r][b];
        }
        if (!ok && lane == 0) { atomicExch(A.status, 7); *(volatile int*)abort_flag = 1; }
        compute_sync();
        if (*(volatile int*)abort_flag) return;
        if (outs) {   // the eight partials of row oi, rhs ob
            C v = ybase;
#pragma unroll
            for (int w = 0; w < 8; ++w) v = cadd(v, part[(w * kMaxRpc + oi) * NB + ob]);
            *yo = v;
        }
        compute_sync();
        if (tid == 0) {
            // this CTA's rows of step s are written (release: ordered after the barrier above);
            // only then are the step's ring slots handed back, so that the refill traffic does
            // not queue in front of the release
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(A.bar) : "memory");
            if (defer)
                for (int i = 0; i < nrow; ++i) mb_arrive(&empty[(g0 + (uint32_t)i) % (uint32_t)R_]);
        }
    }
}

// dst(b,z,k,gc) = [base] + x(b,k,e) on padded columns olo..ohi of the strip
template <typename C>
__global__ void k_slab_out(Geom g, StripDev st, int dir, const C* __restrict__ Y, int ld, double2* __restrict__ dst,
                           const double2* __restrict__ base, int B) {
    const int cofs = st.lo - st.lpml;
    const int olo = st.olo[dir], ohi = min(st.ohi[dir], cofs + st.W - 1), nc = ohi - olo + 1;
    const int64_t tot = (int64_t)B * g.Nz * g.Ny * nc;
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < tot; o += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(o % nc);
        int64_t t = o / nc;
        const int k = (int)(t % g.Ny);
        t /= g.Ny;
        const int z = (int)(t % g.Nz);
        const int b = (int)(t / g.Nz);
        const int gc = olo + i, c = gc - cofs;
        const double2 x = to_d2(Y[((int64_t)b * g.Ny + k) * ld + (int64_t)z * st.W + c]);
        const int64_t idx = (((int64_t)b * g.Nz + z) * g.Ny + k) * g.Nx + gc;
        dst[idx] = base ? cadd(base[idx], x) : x;
    }
}

int grid_for(int64_t work, int threads) {
    const int64_t blocks = (work + threads - 1) / threads;
    return (int)(blocks < 1 ? 1 : (blocks > 152 * 16 ? 152 * 16 : blocks));
}

}  // namespace

// ------------------------------------------------------------------ host
template <typename C>
cudaError_t launch_slab_factor(const Geom& g, const StripDev& st, void* pool, const SlabScratch& sc, int* status,
                               cudaStream_t s, KernelTimer* tm) {
    const int n = st.W * g.Nz;
    if (n > kGjThreads * kGjRowsPerThread) return cudaErrorInvalidValue;
    int dev = 0, nsm = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int nb = imin(nsm, n);
    if ((n + nb - 1) / nb > kGjMaxCols) return cudaErrorInvalidConfiguration;
    // the owned columns stay in shared memory when they fit
    const size_t kCacheMax = 200 * 1024;
    const size_t cache = (size_t)((n + nb - 1) / nb) * n * sizeof(C);
    int cached = cache <= kCacheMax ? 1 : 0;
    size_t dsmem = cached ? cache : 0;
    static bool attr_set = false;
    if (!attr_set) {
        e = cudaFuncSetAttribute(k_gj_invert<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCacheMax);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gj_invert<C>, kGjThreads, dsmem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    C* X = reinterpret_cast<C*>(pool) + st.fac;
    C* M = reinterpret_cast<C*>(sc.M);
    C* mult = reinterpret_cast<C*>(sc.mult);
    const dim3 tiles((n + 31) / 32, (n + 31) / 32), tiles_st((st.ld + 31) / 32, (n + 31) / 32);
    for (int k = 0; k < g.Ny; ++k) {
        {
            TimedLaunch t(tm, "slab_build", s);
            k_slab_build<C><<<tiles, 256, 0, s>>>(g, st, k, k > 0 ? X + (int64_t)(k - 1) * st.bs : nullptr, st.ld,
                                                   M, sc.ldm);
            k_slab_dadd<C><<<(5 * n + 63) / 64, 64, 0, s>>>(g, st, k, M, sc.ldm);
        }
        e = cudaMemsetAsync(sc.bar, 0, 2 * sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
        {
            TimedLaunch t(tm, "slab_gj_invert", s);
            int nn = n, ldm = sc.ldm;
            void* args[] = {&M, &nn, &ldm, (void*)&sc.perm, (void*)&sc.pinv, &mult, (void*)&sc.pivrow,
                            (void*)&sc.bar, &status, &cached};
            e = cudaLaunchCooperativeKernel((const void*)k_gj_invert<C>, dim3(nb), dim3(kGjThreads), args, dsmem, s);
            if (e != cudaSuccess) return e;
        }
        {
            TimedLaunch t(tm, "slab_store", s);
            k_slab_store<C><<<tiles_st, 256, 0, s>>>(M, n, sc.ldm, sc.pinv, X + (int64_t)k * st.bs, st.ld);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename C>
cudaError_t launch_slab_solve(const Geom& g, const StripDev& st, const StripDev* pst, const SweepStep& sp,
                              const SlabWork& wk, const void* pool, cudaStream_t s, KernelTimer* tm) {
    const int n = st.W * g.Nz, Ny = g.Ny, ld = wk.ld, B = wk.B;
    const C* ct = reinterpret_cast<const C*>(g.ct);
    C* Rb = reinterpret_cast<C*>(wk.rbuf);
    C* Y = reinterpret_cast<C*>(wk.ybuf);
    const C* X = reinterpret_cast<const C*>(pool) + st.fac;
    const C* sxz = reinterpret_cast<const C*>(wk.sxz);
    {
        TimedLaunch t(tm, "slab_rhs", s);
        const StripDev pd = pst ? *pst : st;
        k_slab_rhs<C><<<grid_for((int64_t)B * Ny * ld, 256), 256, 0, s>>>(
            g, st, sp, pd, ct, wk.ct_sz, pst ? reinterpret_cast<const C*>(wk.pybuf) : nullptr, ld, Rb, ld, B);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    constexpr int NB = 4;
    int dev = 0, nsm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int rpc = (n + nsm - 1) / nsm, ncta = (n + rpc - 1) / rpc;
    // column segments of 8 per lane up to 2048 unknowns, 16 up to 4096 (complex64 only: the
    // complex128 input vector of 16 columns x 4 right-hand sides would not fit in registers)
    const bool wide = st.ld > 8 * 32 * 8;
    if (rpc > kMaxRpc || st.ld > 8 * 32 * 16 || (wide && sizeof(C) != sizeof(float2))) return cudaErrorInvalidValue;
    const size_t row = (size_t)st.ld * sizeof(C);
    const size_t kSmemMax = 227 * 1024;
    // the kernel for a tile of one or NB right-hand sides
    auto pick = [&](bool one, bool w) -> const void* {
        if constexpr (std::is_same<C, float2>::value) {
            if (w) return one ? (const void*)k_slab_sweep<C, 1, 16> : (const void*)k_slab_sweep<C, NB, 16>;
        }
        return one ? (const void*)k_slab_sweep<C, 1, 8> : (const void*)k_slab_sweep<C, NB, 8>;
    };
    static bool attr_set = false;
    if (!attr_set) {
        for (const void* fn : {pick(true, false), pick(false, false), pick(true, true), pick(false, true)}) {
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
            if (e != cudaSuccess) return e;
        }
        attr_set = true;
    }
    for (int b0 = 0; b0 < B; b0 += NB) {
        const int nb = imin(NB, B - b0);
        const int nbk = nb == 1 ? 1 : NB;
        const size_t fixed = (size_t)8 * kMaxRpc * nbk * sizeof(C) + 128;
        const int ring = (int)std::min<size_t>(64, (kSmemMax - fixed) / (row + 16));
        if (ring < 4) return cudaErrorInvalidValue;   // a row group of the compute warps fits
        const size_t smem = (size_t)ring * row + (size_t)8 * kMaxRpc * nbk * sizeof(C) + (size_t)ring * 16 + 16;
        SlabSweepArgs<C> A{};
        A.X = X;
        A.bs = st.bs;
        A.n = n;
        A.xld = st.ld;
        A.Ny = Ny;
        A.rpc = rpc;
        A.ring = ring;
        A.rhs = Rb + (int64_t)b0 * Ny * ld;
        A.Y = Y + (int64_t)b0 * Ny * ld;
        A.ld = ld;
        A.B = nb;
        A.sxz = sxz;
        A.cyt = ct + g.ct_cy;
        A.bar = wk.bar;
        A.status = wk.status;
        e = cudaMemsetAsync(wk.bar, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
        TimedLaunch t(tm, "slab_sweep", s);
        void* args[] = {&A};
        e = cudaLaunchCooperativeKernel(pick(nbk == 1, wide), dim3(ncta), dim3(kSweepThreads), args, smem, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

template <typename C>
cudaError_t launch_slab_out(const Geom& g, const StripDev& st, int dir, const void* ybuf, int ld, double2* dst,
                            const double2* base, int B, cudaStream_t s, KernelTimer* tm) {
    TimedLaunch t(tm, "slab_out", s);
    const int64_t work = (int64_t)B * g.Nz * g.Ny *
                         (std::min(st.ohi[dir], st.lo - st.lpml + st.W - 1) - st.olo[dir] + 1);
    k_slab_out<C><<<grid_for(work, 256), 256, 0, s>>>(g, st, dir, reinterpret_cast<const C*>(ybuf), ld, dst, base,
                                                     B);
    return cudaGetLastError();
}

template <typename C>
cudaError_t launch_slab_build(const Geom& g, const StripDev& st, int k, const C* Xp, int ld, C* M, int ldm,
                              cudaStream_t s, KernelTimer* tm) {
    const int n = st.W * g.Nz;
    TimedLaunch t(tm, "slab_build", s);
    k_slab_build<C><<<dim3((n + 31) / 32, (n + 31) / 32), 256, 0, s>>>(g, st, k, Xp, ld, M, ldm);
    k_slab_dadd<C><<<(5 * n + 63) / 64, 64, 0, s>>>(g, st, k, M, ldm);
    return cudaGetLastError();
}
template cudaError_t launch_slab_build<float2>(const Geom&, const StripDev&, int, const float2*, int, float2*, int,
                                               cudaStream_t, KernelTimer*);

// Loads this file's module onto the current device (the strip-solve kernels of a
// preconditioner application).
cudaError_t preload_slab_kernels() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_slab_rhs<float2>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_slab_rhs<double2>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_slab_sweep<float2, 1, 8>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_slab_sweep<double2, 1, 8>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_slab_out<float2>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_slab_out<double2>);
    return e;
}

#define HELM_SLAB_INST(C)                                                                                       \
    template cudaError_t launch_slab_factor<C>(const Geom&, const StripDev&, void*, const SlabScratch&, int*,   \
                                               cudaStream_t, KernelTimer*);                                    \
    template cudaError_t launch_slab_solve<C>(const Geom&, const StripDev&, const StripDev*, const SweepStep&, \
                                              const SlabWork&, const void*, cudaStream_t, KernelTimer*);       \
    template cudaError_t launch_slab_out<C>(const Geom&, const StripDev&, int, const void*, int, double2*,     \
                                            const double2*, int, cudaStream_t, KernelTimer*);
HELM_SLAB_INST(float2)
HELM_SLAB_INST(double2)
#undef HELM_SLAB_INST

}  // namespace helm
