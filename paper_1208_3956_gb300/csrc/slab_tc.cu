// Tensor-core factorisation of the dense 3-D strip blocks (Section 2.3, Algorithm 1 on
// strips whose block row is a whole x-z slab), complex64.
//
// Every block X_k = S_k^{-1}, S_k = D_k - C_k X_{k-1} C_k (n x n, n = W N_z), is inverted
// by blocked Gauss-Jordan elimination with partial pivoting, the J strips of the grid side
// by side.  Pivot rows are not exchanged: a row that has served as the pivot of a column is
// marked (kstep) and left out of later pivot searches.  The columns go in panels of kTcBig,
// each made of sub-panels of kTcSub:
//
//   k_tc_panel   (one cluster per strip, the sub-panel's n x kTcSub entries in registers): for
//                each of its columns the largest unused |entry| is the pivot q; the pivot row is
//                scaled by 1/pivot and eliminated from every other row, within the sub-panel.
//                The sub-panel then holds G, its columns of the accumulated row transformation;
//                the kernel also gathers T for the other columns of its panel (below).
//   k_tc_gather  T = the panel's pivot rows as they are, on the columns outside the panel,
//                expanded for the complex product.
//   k_tc_update  every column j to be updated becomes
//                    A(:, j) <- A(:, j) with the source's pivot rows zeroed + G T(:, j),
//                a complex product on the tensor cores: tcgen05.mma kind::tf32 with operands
//                staged in shared memory (inner dimension in chunks of kTcNb complex columns)
//                and the accumulator in tensor memory, each complex64 operand split into a TF32
//                high part and a TF32 remainder (3 products: hi.hi + hi.lo + lo.hi) so that the
//                product keeps complex64 accuracy.  After a sub-panel (the source) it updates the
//                other columns of its panel; after the whole panel (G = the panel's kTcBig
//                columns) every column outside it.
//   k_tc_store   after the last panel the block N holds the inverse up to the pivot order:
//                X(a, c) = N(q_a, pos(c)), q_a the pivot row of step a and pos(c) the step
//                whose pivot row was c; written in the sweep layout of the factor pool.
//
// The complex product uses real operands: a row of G is (Re g_0, Im g_0, Re g_1, ...), and
// complex column j of T gives two B rows, (Re t_0, -Im t_0, Re t_1, ...) for the real part
// and (Im t_0, Re t_0, ...) for the imaginary part, so that the accumulator's columns 2j,
// 2j+1 are the real and imaginary parts of output column j.
#include <climits>

#include "common.cuh"
#include "internal.h"

namespace helm {

namespace {

constexpr int kTcSub = 8;                // sub-panel width (complex columns)
constexpr int kTcNb = 12;                // inner-dimension chunk of an update (complex columns)
constexpr int kTcK = 2 * kTcNb;          // real inner dimension of one chunk (24 = 3 MMAs of 8)
constexpr int kTcBig = 96;               // panel width (complex columns)
constexpr int kTcKT = 2 * kTcBig;        // row length of the T buffer (real)
constexpr int kTcRows = 128;             // rows of an update tile (the MMA's M)
constexpr int kTcCols = 32;              // complex columns of an update tile (N = 64 real)
constexpr int kTcPanelCl = 8;            // CTAs (one cluster) per strip in k_tc_panel
constexpr int kTcPanelThreads = 256;
constexpr int kTcPanelWarps = kTcPanelThreads / 32;
constexpr int kTcPanelRows = 2;          // rows per thread: n <= kTcPanelCl kTcPanelThreads kTcPanelRows = 4096
constexpr int kTcPanelSpan = kTcPanelCl * kTcPanelThreads;   // rows of one sweep over the cluster's threads
constexpr int kTcUpdThreads = 128;
constexpr uint32_t kTcWaitLimit = 1u << 22;
static_assert(kTcBig % kTcSub == 0 && kTcBig % kTcNb == 0 && kTcSub <= kTcNb, "panel geometry");

__device__ __forceinline__ uint32_t tc_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major operand without swizzle: core matrices of 8
// rows x 16 bytes, lbo bytes apart along K, sbo bytes apart between groups of 8 rows.  The
// operands here put element (r, k) of a kTcK-column operand at byte
//     (r / 8) (kTcK / 4) 128 + (k / 4) 128 + (r mod 8) 16 + (k mod 4) 4.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of the tcgen05 family
    return d;
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
    int n, ldm;
    int* qs;       // [n] pivot row of step i
    int* kstep;    // [n] sub-panel in which row r was a pivot row, -1 before
    int* pos;      // [n] step whose pivot row was r
    float* Th;     // [2 npad][kTcKT] the source's pivot rows, expanded (B operand rows; npad: n
    float* Tl;     // rounded up to kTcRows), TF32 high part and remainder
    float2* X;     // the factor pool's block k (row-major, leading dimension xld)
    int xld;
};
constexpr int kTcMaxStrips = 8;
struct TcArgs {
    TcStrip s[kTcMaxStrips];
    int sp;          // k_tc_panel: the sub-panel (columns sp kTcSub ..)
    int glo, ghi;    // gather / update: the source columns (G) and their pivot rows (T)
    int ulo, uhi;    // the columns to update, [ulo, glo) and [ghi, uhi); k_tc_panel: its panel
    int kmin;        // update: rows with kstep >= kmin are the source's pivot rows
    int* status;     // 6: zero or non-finite pivot, 7: a bounded wait gave up
};

// expanded T entries of complex column j, source step t, split into TF32 high part and remainder
__device__ __forceinline__ void tc_put_t(const TcStrip& S, int j, int t, float2 v) {
    const size_t o = (size_t)(2 * j) * kTcKT + 2 * t;
    float h, l;
    tc_split(v.x, h, l);
    S.Th[o] = h;
    S.Tl[o] = l;
    S.Th[o + kTcKT + 1] = h;
    S.Tl[o + kTcKT + 1] = l;
    tc_split(v.y, h, l);
    S.Th[o + kTcKT] = h;
    S.Tl[o + kTcKT] = l;
    S.Th[o + 1] = -h;
    S.Tl[o + 1] = -l;
}

// A warp's pivot candidate for the next column: |entry|^2, its row, and that row's entries in
// the sub-panel's columns (so that the winner's row reaches every thread with the decision).
struct TcCand {
    float best;
    int idx;
    float2 row[kTcSub];
};

__device__ __forceinline__ void tc_cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t tc_cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// address of the same shared variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t tc_mapa(const void* p, uint32_t rank) {
    uint32_t d;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(tc_smem(p)), "r"(rank));
    return d;
}
// 8 bytes into the shared memory of another CTA of the cluster, counted by its mbarrier
__device__ __forceinline__ void tc_st_async(uint32_t addr, uint32_t lo, uint32_t hi, uint32_t mbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.b32 [%0], {%1, %2}, [%3];" ::"r"(addr),
                 "r"(lo), "r"(hi), "r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void tc_arm(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_smem(mbar)), "r"(bytes) : "memory");
}

// One cluster of kTcPanelCl CTAs per strip; thread g = rank kTcPanelThreads + tid of the cluster
// owns rows g + kTcPanelSpan k (k < kTcPanelRows) of the sub-panel in registers.  During step t
// register s holds column (t + s) mod kTcSub (the registers rotate by one column per step, so
// that the loop body indexes them statically).  After the elimination of column t-1 every warp
// sends its candidate for column t, with the candidate row, into every CTA of the cluster
// (st.async, counted by that CTA's mbarrier of the step's buffer); every thread waits for the
// step's kTcPanelCl kTcPanelWarps candidates and reduces them.  No cluster-wide barrier per
// step: a buffer is rewritten two steps later, by senders that have already received this
// CTA's next candidate, which it sends only after reading the buffer.
__global__ void __launch_bounds__(kTcPanelThreads) k_tc_panel(const __grid_constant__ TcArgs a) {
    constexpr int kCands = kTcPanelCl * kTcPanelWarps;
    constexpr uint32_t kStepBytes = kCands * sizeof(TcCand);
    const uint32_t rank = tc_cluster_rank();
    const TcStrip& S = a.s[blockIdx.x / kTcPanelCl];
    const int n = S.n, ldm = S.ldm, c0 = a.sp * kTcSub, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (c0 >= n) return;   // uniform over the cluster
    const int nbp = imin(kTcSub, n - c0);
    const int g = (int)rank * kTcPanelThreads + tid;
    __shared__ __align__(16) TcCand cand[2][kCands];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ int s_q[kTcSub];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tc_arm(&mbar[0], kStepBytes);
        if (nbp > 1) tc_arm(&mbar[1], kStepBytes);
    }
    float2 P[kTcPanelRows][kTcSub];
    bool fr[kTcPanelRows];     // row still free (never a pivot row)
    bool mine[kTcPanelRows];   // row became a pivot row in this sub-panel
#pragma unroll
    for (int k = 0; k < kTcPanelRows; ++k) {
        const int r = g + kTcPanelSpan * k;
        fr[k] = r < n && S.kstep[r] < 0;
        mine[k] = false;
#pragma unroll
        for (int t = 0; t < kTcSub; ++t)
            P[k][t] = (r < n && t < nbp) ? S.M[(int64_t)(c0 + t) * ldm + r] : make_float2(0.f, 0.f);
    }
    tc_cluster_sync();   // every CTA's barriers are armed before the first remote write
    // the warp's candidate for the column at position 0 into cand[buf] of every CTA
    auto propose = [&](int buf) {
        float wb = -1.f;
        int wi = INT_MAX, wk = 0;
#pragma unroll
        for (int k = 0; k < kTcPanelRows; ++k) {
            float v = cabs2(P[k][0]);
            v = v == v ? v : 0.f;   // a NaN entry competes as zero (every free row is a candidate)
            if (fr[k] && v > wb) { wb = v; wi = g + kTcPanelSpan * k; wk = k; }
        }
        // this lane's candidate row, then the warp's winner
        float2 mrow[kTcSub];
#pragma unroll
        for (int s = 0; s < kTcSub; ++s) mrow[s] = P[0][s];
#pragma unroll
        for (int k = 1; k < kTcPanelRows; ++k)
            if (wk == k)
#pragma unroll
                for (int s = 0; s < kTcSub; ++s) mrow[s] = P[k][s];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, wb, o);
            const int oi = __shfl_xor_sync(0xffffffffu, wi, o);
            if (ob > wb || (ob == wb && oi < wi)) { wb = ob; wi = oi; }
        }
        // the winner's row (row r sits in lane r mod 32) to every lane, then lane d < kTcPanelCl
        // sends the candidate to CTA d
        const int wl = wi == INT_MAX ? 0 : (wi & 31);
        float2 row[kTcSub];
#pragma unroll
        for (int s = 0; s < kTcSub; ++s) {
            row[s].x = __shfl_sync(0xffffffffu, mrow[s].x, wl);
            row[s].y = __shfl_sync(0xffffffffu, mrow[s].y, wl);
        }
        if (lane < kTcPanelCl) {
            const uint32_t dst = tc_mapa(&cand[buf][rank * kTcPanelWarps + warp], (uint32_t)lane);
            const uint32_t mb = tc_mapa(&mbar[buf], (uint32_t)lane);
            tc_st_async(dst, __float_as_uint(wb), (uint32_t)wi, mb);
#pragma unroll
            for (int s = 0; s < kTcSub; ++s)
                tc_st_async(dst + 8 + 8 * s, __float_as_uint(row[s].x), __float_as_uint(row[s].y), mb);
        }
    };
    propose(0);
    bool ok = true;
#pragma unroll 1
    for (int t = 0; t < kTcSub; ++t) {
        if (t < nbp && ok) {   // uniform
            uint32_t done = 0;
            for (uint32_t it = 0; it < kTcWaitLimit && !done; ++it)
                asm volatile(
                    "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
                    " selp.u32 %0, 1, 0, p;\n}\n"
                    : "=r"(done)
                    : "r"(tc_smem(&mbar[t & 1])), "r"((uint32_t)((t >> 1) & 1))
                    : "memory");
            // the buffer's next use is armed before any of this CTA's next candidates leave
            if (tid == 0 && done && t + 2 < nbp) tc_arm(&mbar[t & 1], kStepBytes);
            ok = __syncthreads_and(done != 0);   // uniform in the CTA
            if (!ok) {
                if (tid == 0) atomicExch(a.status, 7);
                continue;
            }
            const TcCand* cd = cand[t & 1];
            float bb = -1.f;
            int bx = INT_MAX, bw = 0;
#pragma unroll
            for (int h = 0; h < kCands; h += 32) {
                const float ob = cd[h + lane].best;
                const int oi = cd[h + lane].idx;
                if (ob > bb || (ob == bb && oi < bx)) { bb = ob; bx = oi; bw = h + lane; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, bb, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bx, o);
                const int ow = __shfl_xor_sync(0xffffffffu, bw, o);
                if (ob > bb || (ob == bb && oi < bx)) { bb = ob; bx = oi; bw = ow; }
            }
            if (rank == 0 && tid == 0 && (!(bb > 0.f) || !(bb < INFINITY) || bx >= n))
                atomicExch(a.status, 6);   // zero or non-finite pivot: the result is invalid
            if (bx >= n) { bx = 0; bw = 0; }   // unreachable while a row is free; keeps every index in range
            if (tid == 0) {
                s_q[t] = bx;
                if (rank == 0) S.qs[c0 + t] = bx;
            }
            const float2* prow = cd[bw].row;
            const float2 ip = cinv(prow[0]);
            float2 m[kTcPanelRows];
            bool piv[kTcPanelRows];
#pragma unroll
            for (int k = 0; k < kTcPanelRows; ++k) {
                piv[k] = g + kTcPanelSpan * k == bx;
                m[k] = P[k][0];
                if (piv[k]) { fr[k] = false; mine[k] = true; }
            }
#pragma unroll
            for (int s = 1; s < kTcSub; ++s) {
                const float2 v = cmul(prow[s], ip);
#pragma unroll
                for (int k = 0; k < kTcPanelRows; ++k) P[k][s] = piv[k] ? v : csub(P[k][s], cmul(m[k], v));
            }
#pragma unroll
            for (int k = 0; k < kTcPanelRows; ++k) P[k][0] = piv[k] ? ip : cneg(cmul(m[k], ip));
        }
        // rotate: column t + 1 to position 0 (kTcSub rotations restore the order)
#pragma unroll
        for (int k = 0; k < kTcPanelRows; ++k) {
            const float2 p0 = P[k][0];
#pragma unroll
            for (int s = 0; s + 1 < kTcSub; ++s) P[k][s] = P[k][s + 1];
            P[k][kTcSub - 1] = p0;
        }
        if (t + 1 < nbp && ok) propose((t + 1) & 1);
    }
    // no CTA leaves while a candidate may still be on its way to it
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < kTcPanelRows; ++k) {
        const int r = g + kTcPanelSpan * k;
        if (!ok || r >= n) continue;
#pragma unroll
        for (int t = 0; t < kTcSub; ++t)
            if (t < nbp) S.M[(int64_t)(c0 + t) * ldm + r] = P[k][t];
        if (mine[k]) S.kstep[r] = a.sp;
    }
    // T for the sub-panel's update of the other columns of its panel: the pivot rows at those
    // columns, still untouched by this sub-panel (shared out over the cluster)
    __syncthreads();
    const int plo = a.ulo, phi = imin(a.uhi, n), np = phi - plo;
    if (ok)
        for (int e = g; e < np * kTcSub; e += kTcPanelSpan) {
            const int j = plo + e / kTcSub, t = e % kTcSub;
            if ((j >= c0 && j < c0 + nbp) || t >= nbp) continue;
            tc_put_t(S, j, t, S.M[(int64_t)j * ldm + s_q[t]]);
        }
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The columns to update: [ulo, glo) then [ghi, uhi), at most n.
__device__ __forceinline__ int tc_left(const TcArgs& a) { return a.glo > a.ulo ? a.glo - a.ulo : 0; }

// T for the columns outside the source [glo, ghi): its pivot rows (steps glo .. ghi-1) at each
// column, expanded into the two B rows of the column.
__global__ void k_tc_gather(const __grid_constant__ TcArgs a) {
    const TcStrip& S = a.s[blockIdx.y];
    const int n = S.n, glo = a.glo, ghi = imin(a.ghi, n);
    if (glo >= n) return;
    const int nk = ghi - glo, nl = tc_left(a), nr = imax(imin(a.uhi, n) - ghi, 0);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < (nl + nr) * kTcBig; e += gridDim.x * blockDim.x) {
        const int i = e / kTcBig, t = e % kTcBig;
        const int j = i < nl ? a.ulo + i : ghi + (i - nl);
        tc_put_t(S, j, t, t < nk ? S.M[(int64_t)j * S.ldm + S.qs[glo + t]] : make_float2(0.f, 0.f));
    }
}

// Shared memory of the update tile: one stage of the operands in the core-matrix layout (G
// high and low parts, T high and low parts), an mbarrier and the tensor-memory address slot.
// 36 KB and about 100 registers a thread: five tiles per SM hide each other's load latency.
constexpr uint32_t kTcGBytes = kTcRows * kTcK * 4;        // 12 KB per split part
constexpr uint32_t kTcTBytes = 2 * kTcCols * kTcK * 4;    // 6 KB per split part
constexpr uint32_t kTcStage = 2 * kTcGBytes + 2 * kTcTBytes;
constexpr uint32_t kTcUpdSmem = kTcStage + 64;

__device__ __forceinline__ void tc_sts4(unsigned char* base, uint32_t off, float a, float b, float c, float d) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(tc_smem(base + off)), "f"(a), "f"(b), "f"(c),
                 "f"(d)
                 : "memory");
}

__device__ __forceinline__ bool tc_wait(uint64_t* mbar, uint32_t parity) {
    uint32_t done = 0;
    for (uint32_t it = 0; it < kTcWaitLimit && !done; ++it)
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(tc_smem(mbar)), "r"(parity)
            : "memory");
    return done != 0;
}

// One 128-row x 32-column tile of the update.  Column tiles blockIdx.y < ceil(nl / 32) cover
// [ulo, glo), the others [ghi, uhi).  Thread tid stages row tid of every G chunk and half a B
// row of every T chunk; chunk ch + 1 is read from global memory while the products of chunk ch
// run.  The tile's own entries are read at the start when the source is one chunk (a
// sub-panel: kEarly, three tiles per SM), else while the last products run (a whole panel:
// fewer registers, five tiles per SM).
template <bool kEarly>
__global__ void __launch_bounds__(kTcUpdThreads, kEarly ? 3 : 5) k_tc_update(const __grid_constant__ TcArgs a) {
    extern __shared__ __align__(1024) unsigned char tc_upd_smem[];
    const TcStrip& S = a.s[blockIdx.z];
    const int n = S.n, ldm = S.ldm, glo = a.glo, ghi = imin(a.ghi, n);
    if (glo >= n) return;
    const int nl = tc_left(a), tl_n = (nl + kTcCols - 1) / kTcCols;
    const int y = blockIdx.y;
    const int j0 = y < tl_n ? a.ulo + y * kTcCols : ghi + (y - tl_n) * kTcCols;
    const int jlim = y < tl_n ? glo : imin(a.uhi, n);
    const int r0 = blockIdx.x * kTcRows;
    if (r0 >= n || j0 >= jlim) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(tc_upd_smem + kTcStage);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tc_upd_smem + kTcStage + 16);
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
    const int r = r0 + warp * 32 + lane;
    const int ks = r < n ? S.kstep[r] : -1;
    const bool zero_row = ks >= 0 && ks >= a.kmin;   // a pivot row of the source
    // this thread's row of the tile as it is (the epilogue adds the product to it)
    float2 base[kTcCols];
    auto load_base = [&]() {
#pragma unroll
        for (int e = 0; e < kTcCols; ++e)
            base[e] = (r < n && j0 + e < jlim && !zero_row) ? S.M[(int64_t)(j0 + e) * ldm + r]
                                                            : make_float2(0.f, 0.f);
    };
    if (kEarly) load_base();
    // staging registers: G row tid (kTcNb complex entries), T half row (kTcK / 2 reals, both parts)
    const int nk = ghi - glo, nch = (nk + kTcNb - 1) / kTcNb;
    const int grow = r0 + tid;
    const int brow = tid >> 1, bhalf = tid & 1, bj = j0 + (brow >> 1);
    float2 gv[kTcNb];
    float4 tvh[kTcK / 8], tvl[kTcK / 8];
    auto load = [&](int ch) {
#pragma unroll
        for (int t = 0; t < kTcNb; ++t) {
            const int c = glo + ch * kTcNb + t;
            gv[t] = (c < ghi && grow < n) ? S.M[(int64_t)c * ldm + grow] : make_float2(0.f, 0.f);
        }
        const size_t to = (size_t)(2 * bj + (brow & 1)) * kTcKT + ch * kTcK + bhalf * (kTcK / 2);
#pragma unroll
        for (int i = 0; i < kTcK / 8; ++i) {
            const int t0 = ch * kTcNb + bhalf * (kTcNb / 2) + 2 * i;   // complex source steps t0, t0 + 1
            float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
            if (bj < jlim && t0 < nk) {
                h = *reinterpret_cast<const float4*>(S.Th + to + 4 * i);
                l = *reinterpret_cast<const float4*>(S.Tl + to + 4 * i);
                if (t0 + 1 >= nk) { h.z = h.w = 0.f; l.z = l.w = 0.f; }
            }
            tvh[i] = h;
            tvl[i] = l;
        }
    };
    auto store = [&](unsigned char* st) {
        unsigned char* gh = st;
        unsigned char* gl = gh + kTcGBytes;
        unsigned char* th = gl + kTcGBytes;
        unsigned char* tl = th + kTcTBytes;
        const uint32_t gbase = (uint32_t)((tid >> 3) * (kTcK / 4) * 128 + (tid & 7) * 16);
#pragma unroll
        for (int i = 0; i < kTcNb / 2; ++i) {   // complex entries 2i, 2i+1 = reals 4i .. 4i+3
            float h0, l0, h1, l1, h2, l2, h3, l3;
            tc_split(gv[2 * i].x, h0, l0);
            tc_split(gv[2 * i].y, h1, l1);
            tc_split(gv[2 * i + 1].x, h2, l2);
            tc_split(gv[2 * i + 1].y, h3, l3);
            tc_sts4(gh, gbase + i * 128, h0, h1, h2, h3);
            tc_sts4(gl, gbase + i * 128, l0, l1, l2, l3);
        }
        const uint32_t tbase = (uint32_t)((brow >> 3) * (kTcK / 4) * 128 + (brow & 7) * 16) + bhalf * (kTcK / 8) * 128;
#pragma unroll
        for (int i = 0; i < kTcK / 8; ++i) {
            tc_sts4(th, tbase + i * 128, tvh[i].x, tvh[i].y, tvh[i].z, tvh[i].w);
            tc_sts4(tl, tbase + i * 128, tvl[i].x, tvl[i].y, tvl[i].z, tvl[i].w);
        }
    };
    if (nch > 0) load(0);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    // D f32, A and B tf32, both K-major, N = 64, M = 128
    constexpr uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(2 * kTcCols >> 3) << 17) |
                               ((uint32_t)(kTcRows >> 4) << 24);
    constexpr uint32_t lbo = 128, sbo = (kTcK / 4) * 128;
    bool ok = true;
    for (int ch = 0; ch < nch; ++ch) {
        unsigned char* st = tc_upd_smem;
        // the stage's previous chunk must have been consumed by its products
        const bool free_ok = ch == 0 || tc_wait(mbar, (uint32_t)((ch - 1) & 1));
        store(st);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        ok = __syncthreads_and(free_ok);
        if (!ok) break;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t g_hi = tc_smem(st), g_lo = g_hi + kTcGBytes, t_hi = g_lo + kTcGBytes,
                           t_lo = t_hi + kTcTBytes;
            const uint32_t ga[3] = {g_hi, g_hi, g_lo};
            const uint32_t tb[3] = {t_hi, t_lo, t_hi};
#pragma unroll
            for (int kk = 0; kk < kTcK / 8; ++kk)
#pragma unroll
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
        if (ch + 1 < nch) load(ch + 1);   // in flight while the products run
    }
    if (!kEarly) load_base();   // while the last products run
    // the last commit covers every product issued before it
    if (ok && nch > 0) ok = __syncthreads_and(tc_wait(mbar, (uint32_t)((nch - 1) & 1)));
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
        if (tid == 0) atomicExch(a.status, 7);
    } else {
#pragma unroll
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
            for (int i = 0; i < 8; ++i) {
                const int e = cc / 2 + i, j = j0 + e;
                if (r >= n || j >= jlim) continue;
                S.M[(int64_t)j * ldm + r] =
                    make_float2(base[e].x + __uint_as_float(v[2 * i]), base[e].y + __uint_as_float(v[2 * i + 1]));
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
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.n; i += gridDim.x * blockDim.x) {
        const int q = S.qs[i];
        if (q >= 0 && q < S.n) S.pos[q] = i;
    }
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
        const int c = c0 + i, rr = a0 + tx;
        const int pc = (c < n && rr < n) ? S.pos[c] : -1, q = pc >= 0 ? S.qs[rr] : -1;
        tile[i][tx] = (pc < n && q >= 0 && q < n) ? S.M[(int64_t)pc * S.ldm + q] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const int rr = a0 + i, c = c0 + tx;
        if (rr < n && c < S.xld) S.X[(int64_t)rr * S.xld + c] = tile[tx][i];
    }
}

size_t slab_factor_tc_scratch(int nmax, int ns) {
    const int npad = (nmax + kTcRows - 1) / kTcRows * kTcRows;
    const size_t ldm = (size_t)((nmax + 3) & ~3);
    const size_t per = ldm * nmax * sizeof(float2) + (size_t)3 * nmax * sizeof(int) +
                       (size_t)4 * npad * kTcKT * sizeof(float) + 6 * 256;
    return per * ns;
}

cudaError_t launch_slab_factor_tc(const Geom& g, const StripDev* strips, int ns, void* pool, void* scratch,
                                  int* status, cudaStream_t s, KernelTimer* tm) {
    if (ns < 1 || ns > kTcMaxStrips) return cudaErrorInvalidValue;
    static bool attr_set = false;
    int nmax = 0;
    for (int i = 0; i < ns; ++i) nmax = imax(nmax, strips[i].W * g.Nz);
    if (nmax > kTcPanelSpan * kTcPanelRows) return cudaErrorInvalidValue;   // the block limit
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_tc_update<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcUpdSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_tc_update<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcUpdSmem);
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
        S.M = (float2*)sp; sp += align((size_t)S.ldm * nmax * sizeof(float2));
        S.qs = (int*)sp; sp += align((size_t)nmax * sizeof(int));
        S.kstep = (int*)sp; sp += align((size_t)nmax * sizeof(int));
        S.pos = (int*)sp; sp += align((size_t)nmax * sizeof(int));
        S.Th = (float*)sp; sp += align((size_t)2 * npad_max * kTcKT * sizeof(float));
        S.Tl = (float*)sp; sp += align((size_t)2 * npad_max * kTcKT * sizeof(float));
        S.xld = strips[i].ld;
    }
    const dim3 sgrid((nmax + 3 + 31) / 32, (nmax + 31) / 32, ns);
    float2* pool2 = reinterpret_cast<float2*>(pool);
    // update the columns [ulo, glo) and [ghi, uhi) from the source [glo, ghi)
    auto update = [&](int glo, int ghi, int ulo, int uhi, int kmin, const char* name) {
        A.glo = glo;
        A.ghi = ghi;
        A.ulo = ulo;
        A.uhi = uhi;
        A.kmin = kmin;
        const int nl = imax(glo - ulo, 0), nr = imax(uhi - ghi, 0);
        const int tiles = (nl + kTcCols - 1) / kTcCols + (nr + kTcCols - 1) / kTcCols;
        TimedLaunch t(tm, name, s);
        const dim3 grid(npad_max / kTcRows, tiles, ns);
        if (ghi - glo <= kTcNb)
            k_tc_update<true><<<grid, kTcUpdThreads, kTcUpdSmem, s>>>(A);
        else
            k_tc_update<false><<<grid, kTcUpdThreads, kTcUpdSmem, s>>>(A);
    };
    // k_tc_panel: one cluster of kTcPanelCl CTAs per strip
    cudaLaunchAttribute pattr[1];
    pattr[0].id = cudaLaunchAttributeClusterDimension;
    pattr[0].val.clusterDim.x = kTcPanelCl;
    pattr[0].val.clusterDim.y = 1;
    pattr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t pcfg{};
    pcfg.gridDim = dim3(ns * kTcPanelCl);
    pcfg.blockDim = dim3(kTcPanelThreads);
    pcfg.dynamicSmemBytes = 0;
    pcfg.stream = s;
    pcfg.attrs = pattr;
    pcfg.numAttrs = 1;
    cudaError_t e = cudaSuccess;
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
            for (int s0 = c0; s0 < c1 && e == cudaSuccess; s0 += kTcSub, ++sub) {
                A.sp = sub;
                A.ulo = c0;
                A.uhi = c1;
                {
                    TimedLaunch t(tm, "slab_tc_panel", s);
                    e = cudaLaunchKernelEx(&pcfg, k_tc_panel, A);
                }
                // the sub-panel's transformation on the other columns of its panel (T from the panel kernel)
                if (e == cudaSuccess && c1 - c0 > kTcSub) update(s0, s0 + kTcSub, c0, c1, sub, "slab_tc_update_sub");
                if (e == cudaSuccess) e = cudaGetLastError();
            }
            // the panel's transformation on every column outside it
            if (e == cudaSuccess && nmax > c1 - c0) {
                A.glo = c0;
                A.ghi = c1;
                A.ulo = 0;
                A.uhi = nmax;
                k_tc_gather<<<dim3(((nmax - (c1 - c0)) * kTcBig + 255) / 256, ns), 256, 0, s>>>(A);
                update(c0, c1, 0, nmax, first, "slab_tc_update");
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
