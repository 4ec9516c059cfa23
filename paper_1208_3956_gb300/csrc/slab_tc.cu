// Tensor-core factorisation of the dense 3-D strip blocks (Section 2.3, Algorithm 1 on
// strips whose block row is a whole x-z slab), complex64.
//
// Every block X_k = S_k^{-1}, S_k = D_k - C_k X_{k-1} C_k (n x n, n = W N_z), is inverted
// by blocked Gauss-Jordan elimination with partial pivoting, the J strips of the grid side
// by side.  Pivot rows are not exchanged: a row that has served as the pivot of a column is
// marked (kstep) and left out of later pivot searches.  The columns go in panels of kTcBig,
// each made of sub-panels of kTcNb:
//
//   k_tc_panel   (one CTA per strip, the sub-panel's n x kTcNb entries in shared memory): for
//                each of its columns the largest unused |entry| is the pivot q; the pivot row is
//                scaled by 1/pivot and eliminated from every other row, within the sub-panel.
//                The sub-panel then holds G, its columns of the accumulated row transformation.
//   k_tc_gather  T = the sub-panel's (or panel's) pivot rows as they are, on the columns to be
//                updated, expanded for the complex product.
//   k_tc_update  every column j to be updated becomes
//                    A(:, j) <- A(:, j) with the source's pivot rows zeroed + G T(:, j),
//                a complex product on the tensor cores: tcgen05.mma kind::tf32 with operands
//                staged in shared memory (inner dimension in chunks of kTcNb complex columns)
//                and the accumulator in tensor memory, each complex64 operand split into a TF32
//                high part and a TF32 remainder (3 products: hi.hi + hi.lo + lo.hi) so that the
//                product keeps complex64 accuracy.  After a sub-panel it updates the other
//                columns of its panel; after the whole panel (G = the panel's kTcBig columns)
//                every column outside it.
//   k_tc_store   after the last panel the block N holds the inverse up to the pivot order:
//                X(a, c) = N(q_a, pos(c)), q_a the pivot row of step a and pos(c) the step
//                whose pivot row was c; written in the sweep layout of the factor pool.
//
// The complex product uses real operands: a row of G is (Re g_0, Im g_0, Re g_1, ...), and
// complex column j of T gives two B rows, (Re t_0, -Im t_0, Re t_1, ...) for the real part
// and (Im t_0, Re t_0, ...) for the imaginary part, so that the accumulator's columns 2j,
// 2j+1 are the real and imaginary parts of output column j.
#include "common.cuh"
#include "internal.h"

namespace helm {

namespace {

constexpr int kTcNb = 12;                // sub-panel width (complex columns)
constexpr int kTcK = 2 * kTcNb;          // real inner dimension of one chunk (24 = 3 MMAs of 8)
constexpr int kTcBig = 4 * kTcNb;        // panel width (complex columns)
constexpr int kTcKT = 2 * kTcBig;        // row length of the T buffer (real)
constexpr int kTcRows = 128;             // rows of an update tile (the MMA's M)
constexpr int kTcCols = 32;              // complex columns of an update tile (N = 64 real)
constexpr int kTcPanelThreads = 1024;
constexpr int kTcUpdThreads = 128;
constexpr uint32_t kTcWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t tc_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major operand without swizzle: core matrices of 8
// rows x 16 bytes, lbo bytes apart along K, sbo bytes apart between groups of 8 rows.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of the tcgen05 family
    return d;
}

// byte offset of element (r, k) of a K-major operand with kTcK columns in that layout
__device__ __forceinline__ uint32_t tc_off(int r, int k) {
    return (uint32_t)((r >> 3) * (kTcK / 4) * 128 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

// TF32 keeps the top 19 bits of an FP32 value; hi + lo represents x to about 2^-21
__device__ __forceinline__ void tc_split(float x, float& hi, float& lo) {
    hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
    lo = x - hi;
}

}  // namespace

// One strip's block under inversion and its work arrays.
struct TcStrip {
    float2* M;     // n x n, column-major, leading dimension ldm
    int n, ldm, npad;   // npad: n rounded up to kTcRows
    int* qs;       // [n] pivot row of step i
    int* kstep;    // [n] sub-panel in which row r was a pivot row, -1 before
    int* pos;      // [n] step whose pivot row was r
    float* T;      // [2 npad][kTcKT] the source's pivot rows, expanded (B operand rows)
    float2* X;     // the factor pool's block k (row-major, leading dimension xld)
    int xld;
};
constexpr int kTcMaxStrips = 8;
struct TcArgs {
    TcStrip s[kTcMaxStrips];
    int sp;          // k_tc_panel: the sub-panel (columns sp kTcNb ..)
    int glo, ghi;    // gather / update: the source columns (G) and their pivot rows (T)
    int ulo, uhi;    // gather / update: the columns to update (the source's own skipped)
    int kmin;        // update: rows with kstep >= kmin are the source's pivot rows
    int* status;     // 6: zero or non-finite pivot, 7: a bounded wait gave up
};

__global__ void __launch_bounds__(kTcPanelThreads) k_tc_panel(const __grid_constant__ TcArgs a) {
    extern __shared__ __align__(16) unsigned char tc_panel_smem[];
    const TcStrip& S = a.s[blockIdx.x];
    const int n = S.n, ldm = S.ldm, c0 = a.sp * kTcNb, tid = threadIdx.x;
    if (c0 >= n) return;
    const int nbp = imin(kTcNb, n - c0);
    float2* P = reinterpret_cast<float2*>(tc_panel_smem);   // [kTcNb][n]
    int* ust = reinterpret_cast<int*>(P + (size_t)kTcNb * n); // [n] kstep
    __shared__ float s_best[kTcPanelThreads / 32];
    __shared__ int s_idx[kTcPanelThreads / 32];
    __shared__ int s_q[kTcNb];
    __shared__ float2 s_prow[kTcNb];
    for (int e = tid; e < kTcNb * n; e += kTcPanelThreads) {
        const int t = e / n, r = e % n;
        P[e] = t < nbp ? S.M[(int64_t)(c0 + t) * ldm + r] : make_float2(0.f, 0.f);
    }
    for (int r = tid; r < n; r += kTcPanelThreads) ust[r] = S.kstep[r];
    __syncthreads();
    for (int t = 0; t < nbp; ++t) {
        float best = -1.f;
        int bi = n;
        for (int r = tid; r < n; r += kTcPanelThreads) {
            const float v = cabs2(P[t * n + r]);
            if (ust[r] < 0 && v > best) { best = v; bi = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if ((tid & 31) == 0) { s_best[tid >> 5] = best; s_idx[tid >> 5] = bi; }
        __syncthreads();
        if (tid == 0) {
            float bb = s_best[0];
            int bx = s_idx[0];
            for (int w = 1; w < kTcPanelThreads / 32; ++w)
                if (s_best[w] > bb || (s_best[w] == bb && s_idx[w] < bx)) { bb = s_best[w]; bx = s_idx[w]; }
            if (!(bb > 0.f) || !(bb < INFINITY) || bx >= n) {
                atomicExch(a.status, 6);   // zero or non-finite pivot: the result is invalid
                for (bx = 0; bx < n && ust[bx] >= 0; ++bx) {}
                if (bx >= n) bx = 0;
            }
            ust[bx] = a.sp;
            s_q[t] = bx;
            S.qs[c0 + t] = bx;
        }
        __syncthreads();
        const int q = s_q[t];
        if (tid < nbp) s_prow[tid] = P[tid * n + q];
        __syncthreads();
        const float2 ip = cinv(s_prow[t]);
        for (int r = tid; r < n; r += kTcPanelThreads) {
            const float2 m = P[t * n + r];
            for (int s = 0; s < nbp; ++s) {
                if (s == t) continue;
                const float2 v = cmul(s_prow[s], ip);
                P[s * n + r] = r == q ? v : csub(P[s * n + r], cmul(m, v));
            }
            P[t * n + r] = r == q ? ip : cneg(cmul(m, ip));
        }
        __syncthreads();
    }
    for (int e = tid; e < nbp * n; e += kTcPanelThreads) {
        const int t = e / n, r = e % n;
        S.M[(int64_t)(c0 + t) * ldm + r] = P[e];
    }
    for (int r = tid; r < n; r += kTcPanelThreads) S.kstep[r] = ust[r];
}

// T(j) for the columns j in [ulo, uhi) outside the source [glo, ghi): the source's pivot rows
// (steps glo .. ghi-1) at column j, expanded into the two B rows of complex column j.
__global__ void k_tc_gather(const __grid_constant__ TcArgs a) {
    const TcStrip& S = a.s[blockIdx.y];
    const int n = S.n, glo = a.glo, ghi = imin(a.ghi, n), ulo = a.ulo, uhi = imin(a.uhi, n);
    if (glo >= n) return;
    const int nk = ghi - glo, nj = uhi - ulo;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nj * kTcBig; e += gridDim.x * blockDim.x) {
        const int j = ulo + e / kTcBig, t = e % kTcBig;
        if (j >= glo && j < ghi) continue;
        const float2 v = t < nk ? S.M[(int64_t)j * S.ldm + S.qs[glo + t]] : make_float2(0.f, 0.f);
        float* row_re = S.T + (size_t)(2 * j) * kTcKT;
        float* row_im = row_re + kTcKT;
        row_re[2 * t] = v.x;
        row_re[2 * t + 1] = -v.y;
        row_im[2 * t] = v.y;
        row_im[2 * t + 1] = v.x;
    }
}

// Shared memory of the update tile: the operands in the core-matrix layout, the mbarrier
// and the tensor-memory address slot.
constexpr uint32_t kTcGBytes = kTcRows * kTcK * 4;        // 12 KB per split part
constexpr uint32_t kTcTBytes = 2 * kTcCols * kTcK * 4;    // 6 KB per split part
constexpr uint32_t kTcUpdSmem = 2 * kTcGBytes + 2 * kTcTBytes + 64;

__global__ void __launch_bounds__(kTcUpdThreads) k_tc_update(const __grid_constant__ TcArgs a) {
    extern __shared__ __align__(1024) unsigned char tc_upd_smem[];
    const TcStrip& S = a.s[blockIdx.z];
    const int n = S.n, ldm = S.ldm, glo = a.glo, ghi = imin(a.ghi, n), uhi = imin(a.uhi, n);
    if (glo >= n) return;
    const int r0 = blockIdx.x * kTcRows, j0 = a.ulo + blockIdx.y * kTcCols;
    if (r0 >= n || j0 >= uhi) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* gh = tc_upd_smem;
    unsigned char* gl = gh + kTcGBytes;
    unsigned char* th = gl + kTcGBytes;
    unsigned char* tl = th + kTcTBytes;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(tl + kTcTBytes);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tl + kTcTBytes + 16);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(tslot)),
                     "r"(2 * kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    // D f32, A and B tf32, both K-major, N = 64, M = 128
    constexpr uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(2 * kTcCols >> 3) << 17) |
                               ((uint32_t)(kTcRows >> 4) << 24);
    constexpr uint32_t lbo = 128, sbo = (kTcK / 4) * 128;
    const int nch = (ghi - glo + kTcNb - 1) / kTcNb;
    bool ok = true;
    for (int ch = 0; ch < nch && ok; ++ch) {
        // G chunk: rows r0.., source columns glo + ch kTcNb + t (straight from the block)
        for (int e = tid; e < kTcRows * kTcNb; e += kTcUpdThreads) {
            const int t = e / kTcRows, r = e % kTcRows, c = glo + ch * kTcNb + t;
            const float2 v = (c < ghi && r0 + r < n) ? S.M[(int64_t)c * ldm + r0 + r] : make_float2(0.f, 0.f);
            float hi, lo;
            tc_split(v.x, hi, lo);
            *reinterpret_cast<float*>(gh + tc_off(r, 2 * t)) = hi;
            *reinterpret_cast<float*>(gl + tc_off(r, 2 * t)) = lo;
            tc_split(v.y, hi, lo);
            *reinterpret_cast<float*>(gh + tc_off(r, 2 * t + 1)) = hi;
            *reinterpret_cast<float*>(gl + tc_off(r, 2 * t + 1)) = lo;
        }
        // T chunk: the two B rows of columns j0 .. j0+31
        for (int e = tid; e < 2 * kTcCols * kTcK; e += kTcUpdThreads) {
            const int rr = e / kTcK, k = e % kTcK, j = j0 + rr / 2;
            const bool live = j < uhi && (j < glo || j >= ghi);
            float hi = 0.f, lo = 0.f;
            if (live) tc_split(S.T[(size_t)(2 * j + (rr & 1)) * kTcKT + ch * kTcK + k], hi, lo);
            *reinterpret_cast<float*>(th + tc_off(rr, k)) = hi;
            *reinterpret_cast<float*>(tl + tc_off(rr, k)) = lo;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ga[3] = {tc_smem(gh), tc_smem(gh), tc_smem(gl)};
            const uint32_t tb[3] = {tc_smem(th), tc_smem(tl), tc_smem(th)};
            for (int kk = 0; kk < kTcK / 8; ++kk)
                for (int pr = 0; pr < 3; ++pr) {
                    const uint64_t ad = tc_desc(ga[pr] + kk * 2 * lbo, lbo, sbo);
                    const uint64_t bd = tc_desc(tb[pr] + kk * 2 * lbo, lbo, sbo);
                    const uint32_t acc = (ch > 0 || kk > 0 || pr > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                        : "memory");
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             tc_smem(mbar))
                         : "memory");
        }
        // every thread waits for the chunk's products (its operands are overwritten next)
        uint32_t done = 0;
        for (uint32_t it = 0; it < kTcWaitLimit && !done; ++it)
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(tc_smem(mbar)), "r"((uint32_t)(ch & 1))
                : "memory");
        ok = __syncthreads_and(done != 0);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
        if (tid == 0) atomicExch(a.status, 7);
    } else {
        const int r = r0 + warp * 32 + lane;
        const int ks = r < n ? S.kstep[r] : -1;
        const bool zero_row = ks >= 0 && ks >= a.kmin;   // a pivot row of the source
        for (int cc = 0; cc < 2 * kTcCols; cc += 16) {
            uint32_t v[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int j = j0 + cc / 2 + e;
                if (r >= n || j >= uhi || (j >= glo && j < ghi)) continue;
                float2* dst = S.M + (int64_t)j * ldm + r;
                const float2 base = zero_row ? make_float2(0.f, 0.f) : *dst;
                *dst = make_float2(base.x + __uint_as_float(v[2 * e]), base.y + __uint_as_float(v[2 * e + 1]));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTcCols) : "memory");
}

// pos[q_a] = a
__global__ void k_tc_pos(const __grid_constant__ TcArgs a) {
    const TcStrip& S = a.s[blockIdx.y];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.n; i += gridDim.x * blockDim.x) S.pos[S.qs[i]] = i;
}

// X(a, c) = N(q_a, pos(c)) in the row-major sweep layout (columns n .. xld-1 zero).
__global__ void __launch_bounds__(256) k_tc_store(const __grid_constant__ TcArgs a) {
    __shared__ float2 tile[32][33];
    const TcStrip& S = a.s[blockIdx.z];
    const int n = S.n;
    const int a0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    if (a0 >= n || c0 >= S.xld) return;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int i = ty; i < 32; i += 8) {   // column c0+i of X, rows a0+tx
        const int c = c0 + i, r = a0 + tx;
        tile[i][tx] = (c < n && r < n) ? S.M[(int64_t)S.pos[c] * S.ldm + S.qs[r]] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const int r = a0 + i, c = c0 + tx;
        if (r < n && c < S.xld) S.X[(int64_t)r * S.xld + c] = tile[tx][i];
    }
}

size_t slab_factor_tc_scratch(int nmax, int ns) {
    const int npad = (nmax + kTcRows - 1) / kTcRows * kTcRows;
    const size_t ldm = (size_t)((nmax + 3) & ~3);
    const size_t per = ldm * nmax * sizeof(float2) + (size_t)3 * nmax * sizeof(int) +
                       (size_t)2 * npad * kTcKT * sizeof(float) + 4 * 256;
    return per * ns;
}

cudaError_t launch_slab_factor_tc(const Geom& g, const StripDev* strips, int ns, void* pool, void* scratch,
                                  int* status, cudaStream_t s, KernelTimer* tm) {
    if (ns < 1 || ns > kTcMaxStrips) return cudaErrorInvalidValue;
    static bool attr_set = false;
    int nmax = 0;
    for (int i = 0; i < ns; ++i) nmax = imax(nmax, strips[i].W * g.Nz);
    const size_t psmem = (size_t)kTcNb * nmax * sizeof(float2) + (size_t)nmax * sizeof(int);
    if (psmem > 220 * 1024) return cudaErrorInvalidValue;   // n <= 2048 (the block limit)
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_tc_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_tc_update, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcUpdSmem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    TcArgs A{};
    A.status = status;
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    char* sp = (char*)scratch;
    const int npad_max = (nmax + kTcRows - 1) / kTcRows * kTcRows;
    for (int i = 0; i < ns; ++i) {
        TcStrip& S = A.s[i];
        S.n = strips[i].W * g.Nz;
        S.ldm = (nmax + 3) & ~3;
        S.npad = (S.n + kTcRows - 1) / kTcRows * kTcRows;
        S.M = (float2*)sp; sp += align((size_t)S.ldm * nmax * sizeof(float2));
        S.qs = (int*)sp; sp += align((size_t)nmax * sizeof(int));
        S.kstep = (int*)sp; sp += align((size_t)nmax * sizeof(int));
        S.pos = (int*)sp; sp += align((size_t)nmax * sizeof(int));
        S.T = (float*)sp; sp += align((size_t)2 * npad_max * kTcKT * sizeof(float));
        S.xld = strips[i].ld;
    }
    const dim3 sgrid((nmax + 3 + 31) / 32, (nmax + 31) / 32, ns);
    float2* pool2 = reinterpret_cast<float2*>(pool);
    cudaError_t e = cudaSuccess;
    // gather T, then update the columns [ulo, uhi) from the source [glo, ghi)
    auto source_update = [&](int glo, int ghi, int ulo, int uhi, int kmin) {
        A.glo = glo;
        A.ghi = ghi;
        A.ulo = ulo;
        A.uhi = uhi;
        A.kmin = kmin;
        const int nj = uhi - ulo;
        k_tc_gather<<<dim3((nj * kTcBig + 255) / 256, ns), 256, 0, s>>>(A);
        TimedLaunch t(tm, "slab_tc_update", s);
        k_tc_update<<<dim3(npad_max / kTcRows, (nj + kTcCols - 1) / kTcCols, ns), kTcUpdThreads, kTcUpdSmem, s>>>(A);
    };
    for (int k = 0; k < g.Ny && e == cudaSuccess; ++k) {
        for (int i = 0; i < ns && e == cudaSuccess; ++i) {
            const StripDev& st = strips[i];
            A.s[i].X = pool2 + st.fac + (int64_t)k * st.bs;
            e = launch_slab_build<float2>(g, st, k, k > 0 ? pool2 + st.fac + (int64_t)(k - 1) * st.bs : nullptr,
                                          st.ld, A.s[i].M, A.s[i].ldm, s, tm);
            if (e == cudaSuccess) e = cudaMemsetAsync(A.s[i].kstep, 0xFF, (size_t)A.s[i].n * sizeof(int), s);
        }
        int sub = 0;
        for (int c0 = 0; c0 < nmax && e == cudaSuccess; c0 += kTcBig) {
            const int c1 = imin(c0 + kTcBig, nmax), first = sub;
            for (int s0 = c0; s0 < c1 && e == cudaSuccess; s0 += kTcNb, ++sub) {
                A.sp = sub;
                {
                    TimedLaunch t(tm, "slab_tc_panel", s);
                    k_tc_panel<<<ns, kTcPanelThreads, psmem, s>>>(A);
                }
                // the sub-panel's transformation on the other columns of its panel
                if (c1 - c0 > kTcNb) source_update(s0, s0 + kTcNb, c0, c1, sub);
                e = cudaGetLastError();
            }
            // the panel's transformation on every column outside it
            if (e == cudaSuccess && nmax > c1 - c0) {
                if (c0 > 0) source_update(c0, c1, 0, c0, first);
                if (c1 < nmax) source_update(c0, c1, c1, nmax, first);
                e = cudaGetLastError();
            }
        }
        if (e != cudaSuccess) break;
        k_tc_pos<<<dim3(8, ns), 256, 0, s>>>(A);
        {
            TimedLaunch t(tm, "slab_tc_store", s);
            k_tc_store<<<sgrid, 256, 0, s>>>(A);
        }
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace helm
