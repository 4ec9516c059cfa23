// One strip solve of the double sweep (Section 2.1, Eqs. solve_upward and
// solve_downward) on the partitioned block-tridiagonal factors of factor.cu.
//
// k_sweep_chunk (grid: chunks x RHS tiles)
//   * builds the strip right-hand side S^(j) r for every row of its chunk
//     (masked source plus the single-layer-potential transfer on two columns);
//   * streams the chunk's Sinv_k blocks global -> shared memory with TMA bulk
//     copies (cp.async.bulk + mbarrier ring; the whole chunk stays resident when
//     it fits, so the back substitution reads no HBM);
//   * runs the chain z_k = Sinv_k (b_k - C_k z_{k-1}), x_k = z_k - Sinv_k C_{k+1} x_{k+1}
//     with the W x W products split over the warps (lanes own rows);
//   * adds its two parts of the separator right-hand sides, Rinv_q times
//     (b_s - C_s y_q(last)) and -Rinv_q C_{s+1} y_{q+1}(first);
//   * the last chunk CTA of a separator group to finish (atomic arrival
//     counter per group, no waiting) solves the group's separators with the
//     level-2 separators held at zero (twisted chain z_i = a_i - E_i z_outer,
//     x_i = z_i - F_i x_inner) and adds the group's parts of the level-2
//     right-hand sides; the last group to finish solves the level-2 system.
// k_sweep_sepfix (grid: separators x RHS tiles; only with more than one group)
//   x_q = y_q - GT2_q x2_above - GB2_q x2_below for the grouped separators.
// k_sweep_correct (grid: rows x RHS tiles)
//   x_k = y_k - GT_p(k) x_{p-1} - GB_p(k) x_p on the output columns only, scatter
//   to the output field (compose) and emit the transfer difference.
//
// Every mbarrier wait is bounded; on time-out the kernel records
// HELM_ETIMEOUT in the status word, drains its copies (bounded) and returns.
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace helm {

static constexpr int kMaxRing = 32;
static constexpr uint32_t kWaitLimit = 1u << 22;
static constexpr int kParts = 4;   // separator right-hand-side parts: 2 from chunks, 2 from groups

// load-order table entries: factor pool << 24 | block index in that pool
enum : int { kSinv = 0, kRinv = 1, kEo = 2, kFi = 3, kP2L = 4, kP2U = 5 };
__host__ __device__ constexpr int enc(int pool, int idx) { return (pool << 24) | idx; }

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* m) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(m))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(m)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* m, uint32_t parity) {
    for (uint32_t it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(m, parity)) return true;
    return false;
}

// ------------------------------------------------------------------ args
struct SweepArgs {
    Geom g;
    StripDev st;
    SweepStep sp;
    int Wmax, B, Bt;
    int ring;                // slots of the block ring
    int zrows;               // rows of the z buffer (max chunk rows, separators)
    uint32_t slot_bytes;     // bytes of one staged W x W block
    const void* Sinv;
    const void* Rinv;
    const void* E;
    const void* F;
    const void* P2L;         // level-2 products Rinv2 L, Rinv2 U (null with one group)
    const void* P2U;
    void* ybuf;              // [B][Ny][Wmax] chunk solutions, then separator values
    void* parts;             // [B][P-1][kParts][Wmax] separator right-hand-side parts
    int* counters;           // [ntile][G+1] arrival counters, left at zero
    int* status;
};

template <typename C>
__device__ __forceinline__ const C* ctab(const Geom& g) { return reinterpret_cast<const C*>(g.ct); }

template <typename C>
__device__ __forceinline__ C coupling(const SweepArgs& A, int k, int c) {
    return cmul(ctab<C>(A.g)[A.st.ctab + c], ctab<C>(A.g)[A.g.ct_cy + k]);
}

// S^(j) r at strip-local column c, row k, RHS b (working precision)
template <typename C>
__device__ __forceinline__ C rhs_entry(const SweepArgs& A, int k, int c, int b) {
    const int gc = A.st.lo - A.st.lpml + c;
    double2 v = make_double2(0.0, 0.0);
    const int64_t row = (int64_t)b * A.g.Ny + k;
    if (gc >= A.sp.mlo && gc <= A.sp.mhi) v = A.sp.src[row * A.g.Nx + gc];
    if (A.sp.tin && (gc == A.sp.t0 || gc == A.sp.t0 + 1)) {
        const double2 t = A.sp.tin[row];
        v.x = fma(A.sp.tcoef, t.x, v.x);
        v.y = fma(A.sp.tcoef, t.y, v.y);
    }
    return cmul(CT<C>::from(v), cmul(ctab<C>(A.g)[A.st.ctab + c], ctab<C>(A.g)[A.g.ct_sy + k]));
}

template <typename C>
__device__ __forceinline__ C* yrow(const SweepArgs& A, int b, int k) {
    return reinterpret_cast<C*>(A.ybuf) + ((int64_t)b * A.g.Ny + k) * A.Wmax;
}

// Shared-memory carve-up (bytes), identical on host and device.
struct SweepSmem {
    uint32_t slots, zb, tv, cx, cy, order, mbar, flags, total;
};
__host__ __device__ inline SweepSmem sweep_smem(int ring, uint32_t slot_bytes, int zrows, int Bt, int W,
                                                int esz) {
    SweepSmem s;
    uint32_t o = 0;
    s.slots = o; o += ring * slot_bytes;
    s.zb = o; o += ((uint32_t)zrows * Bt * W * esz + 15u) & ~15u;
    s.tv = o; o += 4u * Bt * 64 * esz;                         // in/out vectors of both chains
    s.cx = o; o += 64u * esz;
    s.cy = o; o += ((uint32_t)(zrows + 2) * esz + 15u) & ~15u;
    s.order = o; o += ((uint32_t)(2 * zrows + 4) * 4 + 15u) & ~15u;   // load order table
    s.mbar = o; o += kMaxRing * 8;
    s.flags = o; o += 16;
    s.total = o;
    return s;
}

// ------------------------------------------------------------------ chunk + separators
// Products of one chain step.  The CTA has ceil(W/8) warps; lane l of warp w
// owns row r = 8w + l/4 (clamped to W-1 for the idle rows of the last warp) and
// the NJ contiguous columns g*NJ .. g*NJ+NJ-1, g = l%4, of a sweep-layout block
// (row-major, leading dimension 4 NJ + 2, zero beyond column W).  Both the
// factor row and the vector are read as 16-byte runs; two xor shuffles finish
// the row sums on all four lanes of the row.
__device__ __forceinline__ void load_run2(float2* v, const float2* p, int n) {
    for (int jj = 0; jj < n / 2; ++jj) {
        const float4 q = reinterpret_cast<const float4*>(p)[jj];
        v[2 * jj] = make_float2(q.x, q.y);
        v[2 * jj + 1] = make_float2(q.z, q.w);
    }
}
__device__ __forceinline__ void load_run2(double2* v, const double2* p, int n) {
    for (int j = 0; j < n; ++j) v[j] = p[j];
}
template <typename C, int NJ>
__device__ __forceinline__ void load_row(C (&v)[NJ], const C* p) {
#pragma unroll
    for (int j = 0; j < NJ; j += 2) load_run2(&v[j], p + j, 2);
}
template <typename C, int NJ>
__device__ __forceinline__ C row_dot(const C (&s)[NJ], const C* t) {
    C tv[NJ];
    load_row<C, NJ>(tv, t);
    C a0 = CT<C>::zero(), a1 = CT<C>::zero();
#pragma unroll
    for (int j = 0; j < NJ; j += 2) {
        a0 = cfma(s[j], tv[j], a0);
        a1 = cfma(s[j + 1], tv[j + 1], a1);
    }
    C v = cadd(a0, a1);
    v.x += __shfl_xor_sync(0xffffffffu, v.x, 1);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, 1);
    v.x += __shfl_xor_sync(0xffffffffu, v.x, 2);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, 2);
    return v;
}

// Both chains of a step in one instruction stream: vd[b] = Sd-row . td_b and
// vu[b] = Su-row . tu_b (the row sums complete on all four lanes of a row).
// D / U select the active chains at compile time.
template <typename C, int NJ, int BT, bool D, bool U>
__device__ __forceinline__ void dual_rows(const C* __restrict__ Sd, const C* __restrict__ td,
                                          const C* __restrict__ Su, const C* __restrict__ tu, int nb,
                                          C (&vd)[BT], C (&vu)[BT]) {
    C sd[NJ], su[NJ];
    if (D) load_row<C, NJ>(sd, Sd);
    if (U) load_row<C, NJ>(su, Su);
#pragma unroll
    for (int b = 0; b < BT; ++b) {
        if (b < nb) {
            C xd[NJ], xu[NJ];
            if (D) load_row<C, NJ>(xd, td + b * 64);
            if (U) load_row<C, NJ>(xu, tu + b * 64);
            C d0 = CT<C>::zero(), d1 = CT<C>::zero(), u0 = CT<C>::zero(), u1 = CT<C>::zero();
#pragma unroll
            for (int j = 0; j < NJ; j += 2) {
                if (D) { d0 = cfma(sd[j], xd[j], d0); d1 = cfma(sd[j + 1], xd[j + 1], d1); }
                if (U) { u0 = cfma(su[j], xu[j], u0); u1 = cfma(su[j + 1], xu[j + 1], u1); }
            }
            C a = cadd(d0, d1), c = cadd(u0, u1);
#pragma unroll
            for (int o = 1; o <= 2; o <<= 1) {
                if (D) { a.x += __shfl_xor_sync(0xffffffffu, a.x, o); a.y += __shfl_xor_sync(0xffffffffu, a.y, o); }
                if (U) { c.x += __shfl_xor_sync(0xffffffffu, c.x, o); c.y += __shfl_xor_sync(0xffffffffu, c.y, o); }
            }
            vd[b] = a;
            vu[b] = c;
        }
    }
}
template <typename C, int NJ, int BT>
__device__ __forceinline__ void dual_dispatch(bool dn, bool up, const C* Sd, const C* td, const C* Su,
                                              const C* tu, int nb, C (&vd)[BT], C (&vu)[BT]) {
    if (dn && up) dual_rows<C, NJ, BT, true, true>(Sd, td, Su, tu, nb, vd, vu);
    else if (dn) dual_rows<C, NJ, BT, true, false>(Sd, td, Su, tu, nb, vd, vu);
    else if (up) dual_rows<C, NJ, BT, false, true>(Sd, td, Su, tu, nb, vd, vu);
}

// The CTA is ceil(W/8) compute warps plus one producer warp.  The producer's
// lane 0 owns the TMA ring: it initialises the barriers, issues every bulk
// copy, and right after each step's barrier refills the slots that step
// consumed, while the compute warps already run the next step.
template <typename C, int NJ, int BT>
__global__ void __launch_bounds__(288) k_sweep_chunk(SweepArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int LD = 4 * NJ + 2;
    const int W = A.st.W;
    const int esz = (int)sizeof(C);
    const SweepSmem L = sweep_smem(A.ring, A.slot_bytes, A.zrows, BT, W, esz);
    unsigned char* slots = smem + L.slots;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L.mbar);
    C* zb = reinterpret_cast<C*>(smem + L.zb);       // [zrows][BT][W]
    C* v0 = reinterpret_cast<C*>(smem + L.tv);       // four [BT][64] vectors: in/out of both chains
    C* vin_d = v0;
    C* vin_u = v0 + BT * 64;
    C* vout_d = v0 + 2 * BT * 64;
    C* vout_u = v0 + 3 * BT * 64;
    C* csx = reinterpret_cast<C*>(smem + L.cx);      // s_x(c)
    C* ccy = reinterpret_cast<C*>(smem + L.cy);      // -alpha_y(k-1/2)/h^2, k = r0..r1
    int* order = reinterpret_cast<int*>(smem + L.order);
    volatile int* flags = reinterpret_cast<int*>(smem + L.flags);
    const int p = blockIdx.x, tile = blockIdx.y;
    const int b0 = tile * BT;
    const int nb = imin(BT, A.B - b0);
    const int r0 = A.g.r0[p], r1 = A.g.r1[p], m = r1 - r0;
    const int t = r0 + (m - 1) / 2;                  // twist row
    const int nd = t - r0, nu = r1 - 1 - t, nmx = imax(nd, nu);
    const int P = A.g.P, Q = P - 1;
    const int tid = threadIdx.x;
    const int ptid = blockDim.x - 32;                // the producer thread
    const bool producer = tid == ptid;
    const bool compute = tid < ptid;
    const int64_t bs = A.st.bs;
    const int ring = A.ring;
    const uint32_t sb = A.slot_bytes;
    const C* Sinv = reinterpret_cast<const C*>(A.Sinv) + A.st.fac;
    const C* Rinv = reinterpret_cast<const C*>(A.Rinv) + A.st.red;
    const C* Eb = reinterpret_cast<const C*>(A.E) + A.st.red;
    const C* Fb = reinterpret_cast<const C*>(A.F) + A.st.red;
    const C* P2Lb = A.P2L ? reinterpret_cast<const C*>(A.P2L) + A.st.red : nullptr;
    const C* P2Ub = A.P2U ? reinterpret_cast<const C*>(A.P2U) + A.st.red : nullptr;
    const bool resident = ring >= m + 2;
    const bool has_below = p < P - 1, has_above = p > 0;
    // ---- load order of the chunk phase (rows of Sinv, then Rinv below / above)
    //   forward: s = 0..nmx-1: down row r0+s, up row r1-1-s; then the twist row
    //   back (streaming only): s = 0..nmx-1: down row t-1-s, up row t+1+s
    const int nload = m + (resident ? 0 : m - 1) + (has_below ? 1 : 0) + (has_above ? 1 : 0);
    // ---- ring state: load G lives in slot G % ring and completes phase (G / ring) & 1
    int issued = 0, consumed = 0;           // issued: the producer's count
    int cslot = 0;
    uint32_t cpar = 0;
    int rf = 0, rfslot = 0;                 // producer: next consumed load whose slot is reused
    int nseq = nload;                       // loads in the current sequence
    int seqbase = 0;                        // first load number of the current sequence
    bool sep_phase = false;
    auto src_of = [&](int G) -> const C* {
        const int e = order[G - seqbase];
        const int64_t o = (int64_t)(e & 0xffffff) * bs;
        switch (e >> 24) {
            case kSinv: return Sinv + o;
            case kRinv: return Rinv + o;
            case kEo: return Eb + o;
            case kFi: return Fb + o;
            case kP2L: return P2Lb + o;
            default: return P2Ub + o;
        }
    };
    auto issue_into = [&](int slot, const C* src) {   // producer only
        uint64_t* mb = &mbar[slot];
        fence_proxy_async();
        mbar_expect_tx(mb, sb);
        bulk_g2s(slots + (size_t)slot * sb, src, sb, mb);
        ++issued;
    };
    auto consume = [&]() -> const C* {
        const C* S = reinterpret_cast<const C*>(slots + (size_t)cslot * sb);
        if (compute && !mbar_wait(&mbar[cslot], cpar)) flags[1] = 1;
        ++consumed;
        if (++cslot == ring) { cslot = 0; cpar ^= 1u; }
        return S;
    };
    // producer, after a barrier: every consumed slot is free; reuse it
    auto refill = [&]() {
        while (rf < consumed) {
            if (rf + ring < nseq) issue_into(rfslot, src_of(rf + ring));
            ++rf;
            if (++rfslot == ring) rfslot = 0;
        }
    };
    auto drain = [&]() {
        if (producer) {
            atomicExch(A.status, 7);
            for (int Gd = consumed - 1; Gd < issued; ++Gd)
                if (Gd >= 0) mbar_wait(&mbar[Gd % ring], (uint32_t)((Gd / ring) & 1));
        }
        __syncthreads();
    };
    if (producer) {
        int G = 0;
        for (int s = 0; s < nmx; ++s) {
            if (s < nd) order[G++] = enc(kSinv, r0 + s);
            if (s < nu) order[G++] = enc(kSinv, r1 - 1 - s);
        }
        order[G++] = enc(kSinv, t);
        if (!resident)
            for (int s = 0; s < nmx; ++s) {
                if (s < nd) order[G++] = enc(kSinv, t - 1 - s);
                if (s < nu) order[G++] = enc(kSinv, t + 1 + s);
            }
        if (has_below) order[G++] = enc(kRinv, p);
        if (has_above) order[G++] = enc(kRinv, p - 1);
        flags[1] = 0;
        for (int i = 0; i < ring; ++i) mbar_init(&mbar[i], 1);
        fence_mbar_init();
        for (int i = 0; i < imin(ring, nload); ++i) issue_into(i, src_of(i));
    }
    const C* ct = ctab<C>(A.g);
    for (int o = tid; o < 4 * BT * 64; o += blockDim.x) v0[o] = CT<C>::zero();
    for (int c = tid; c < W; c += blockDim.x) csx[c] = ct[A.st.ctab + c];
    for (int k = r0 + tid; k <= r1; k += blockDim.x) ccy[k - r0] = ct[A.g.ct_cy + k];
    __syncthreads();
    // right-hand sides of every chunk row (independent of the chain)
    for (int o = tid; o < m * nb * W; o += blockDim.x) {
        const int c = o % W, b = (o / W) % nb, r = o / (W * nb);
        const C v = rhs_entry<C>(A, r0 + r, c, b0 + b);
        zb[(r * BT + b) * W + c] = v;
        if (r == 0 && nd > 0) vin_d[b * 64 + c] = v;            // down chain starts at r0
        if (r == m - 1 && nu > 0) vin_u[b * 64 + c] = v;        // up chain starts at r1-1
    }
    // per-lane geometry
    const int w = tid >> 5, l = tid & 31;
    const int row = w * 8 + (l >> 2);
    const int g = l & 3;
    const bool rowok = compute && row < W;
    const int rc = imin(row, W - 1);
    const int lofs = rc * LD + g * NJ;     // this lane's run inside a block
    const int vofs = g * NJ;               // ... and inside a vector
    const C csx_r = csx[rc];
    __syncthreads();
    auto zr = [&](int k) -> C* { return zb + (k - r0) * BT * W; };   // row k, b = 0
    auto cpl = [&](int k) -> C { return cmul(csx_r, ccy[k - r0]); }; // C_k at this lane's row
    auto finish = [&]() -> bool {
        __syncthreads();
        if (flags[1]) { drain(); return false; }
        if (producer && !(resident && !sep_phase)) refill();
        C* x = vin_d; vin_d = vout_d; vout_d = x;
        x = vin_u; vin_u = vout_u; vout_u = x;
        return true;
    };
    C vd[BT], vu[BT];
    const bool own1 = rowok && g == 0;                 // BT = 1: the lane that stores a row
    auto owns = [&](int b) -> bool { return BT == 1 ? own1 : (b < nb && rowok && (b & 3) == g); };
    C* const zl = zb + row;                            // this lane's entry of z-buffer row r0, b = 0
    const int zs = BT * W;                             // z-buffer stride between grid rows
    // ---- forward elimination: both halves while both have rows, then the longer one
    auto fwd = [&](auto Dc, auto Uc, int s) -> bool {
        constexpr bool D = decltype(Dc)::value, U = decltype(Uc)::value;
        const C* Sd = D ? consume() : nullptr;
        const C* Su = U ? consume() : nullptr;
        if (compute) dual_rows<C, NJ, BT, D, U>(Sd + lofs, vin_d + vofs, Su + lofs, vin_u + vofs, nb, vd, vu);
        if (D) {   // z_kd, kd = r0+s; next down input b_{kd+1} - C_{kd+1} z_kd (if kd+1 < t)
            const C ck = cmul(csx_r, ccy[s + 1]);
            C* zp = zl + s * zs;
            const bool more = r0 + s + 1 < t;
#pragma unroll
            for (int b = 0; b < BT; ++b)
                if (owns(b)) {
                    zp[b * W] = vd[b];
                    if (more) vout_d[b * 64 + row] = csub(zp[zs + b * W], cmul(ck, vd[b]));
                }
        }
        if (U) {   // z_ku, ku = r1-1-s; next up input b_{ku-1} - C_ku z_ku (if ku-1 > t)
            const int ui = m - 1 - s;                      // ku - r0
            const C ck = cmul(csx_r, ccy[ui]);
            C* zp = zl + ui * zs;
            const bool more = r1 - 2 - s > t;
#pragma unroll
            for (int b = 0; b < BT; ++b)
                if (owns(b)) {
                    zp[b * W] = vu[b];
                    if (more) vout_u[b * 64 + row] = csub(zp[-zs + b * W], cmul(ck, vu[b]));
                }
        }
        return finish();
    };
    {
        int s = 0;
        const int nboth = imin(nd, nu);
        for (; s < nboth; ++s)
            if (!fwd(std::true_type{}, std::true_type{}, s)) return;
        for (; s < nd; ++s)
            if (!fwd(std::true_type{}, std::false_type{}, s)) return;
        for (; s < nu; ++s)
            if (!fwd(std::false_type{}, std::true_type{}, s)) return;
    }
    // ---- twist row: y_t = Sinv_t (b_t - C_t z_{t-1} - C_{t+1} z_{t+1})
    for (int o = tid; o < nb * W; o += blockDim.x) {
        const int c = o % W, b = o / W;
        C v = zr(t)[b * W + c];
        if (nd > 0) v = csub(v, cmul(cmul(csx[c], ccy[t - r0]), zr(t - 1)[b * W + c]));
        if (nu > 0) v = csub(v, cmul(cmul(csx[c], ccy[t + 1 - r0]), zr(t + 1)[b * W + c]));
        vin_d[b * 64 + c] = v;
    }
    __syncthreads();
    {
        const C* St = consume();
        if (compute) dual_rows<C, NJ, BT, true, false>(St + lofs, vin_d + vofs, St, vin_u, nb, vd, vu);
        const C cd = cpl(t), cu = cpl(t + 1);
#pragma unroll
        for (int b = 0; b < BT; ++b)
            if (owns(b)) {
                zr(t)[b * W + row] = vd[b];
                vout_d[b * 64 + row] = cmul(cd, vd[b]);   // C_t y_t for row t-1
                vout_u[b * 64 + row] = cmul(cu, vd[b]);   // C_{t+1} y_t for row t+1
            }
        if (!finish()) return;
    }
    // ---- outward back substitution: y_k = z_k - Sinv_k C y_inner
    auto bwd = [&](auto Dc, auto Uc, int s) -> bool {
        constexpr bool D = decltype(Dc)::value, U = decltype(Uc)::value;
        const int di = nd - 1 - s;              // kd - r0, kd = t-1-s
        const int ui = nd + 1 + s;              // ku - r0, ku = t+1+s
        const C* Sd = nullptr;
        const C* Su = nullptr;
        if (resident) {
            // forward position: down row r0+i at i + min(i, nu); up row r1-1-i at min(i+1, nd) + i
            if (D) Sd = reinterpret_cast<const C*>(slots + (size_t)(di + imin(di, nu)) * sb);
            if (U) { const int i = m - 1 - ui; Su = reinterpret_cast<const C*>(slots + (size_t)(imin(i + 1, nd) + i) * sb); }
        } else {
            if (D) Sd = consume();
            if (U) Su = consume();
        }
        if (compute) dual_rows<C, NJ, BT, D, U>(Sd + lofs, vin_d + vofs, Su + lofs, vin_u + vofs, nb, vd, vu);
        if (D) {
            const C ck = cmul(csx_r, ccy[di]);      // C_kd y_kd for row kd-1
            C* zp = zl + di * zs;
#pragma unroll
            for (int b = 0; b < BT; ++b)
                if (owns(b)) {
                    const C y = csub(zp[b * W], vd[b]);
                    zp[b * W] = y;
                    vout_d[b * 64 + row] = cmul(ck, y);
                }
        }
        if (U) {
            const C ck = cmul(csx_r, ccy[ui + 1]);  // C_{ku+1} y_ku for row ku+1
            C* zp = zl + ui * zs;
#pragma unroll
            for (int b = 0; b < BT; ++b)
                if (owns(b)) {
                    const C y = csub(zp[b * W], vu[b]);
                    zp[b * W] = y;
                    vout_u[b * 64 + row] = cmul(ck, y);
                }
        }
        return finish();
    };
    {
        int s = 0;
        const int nboth = imin(nd, nu);
        for (; s < nboth; ++s)
            if (!bwd(std::true_type{}, std::true_type{}, s)) return;
        for (; s < nd; ++s)
            if (!bwd(std::true_type{}, std::false_type{}, s)) return;
        for (; s < nu; ++s)
            if (!bwd(std::false_type{}, std::true_type{}, s)) return;
    }
    // ---- chunk solution to global memory
    for (int o = tid; o < m * nb * W; o += blockDim.x) {
        const int c = o % W, b = (o / W) % nb, r = o / (W * nb);
        yrow<C>(A, b0 + b, r0 + r)[c] = zb[(r * BT + b) * W + c];
    }
    // ---- separator right-hand-side parts, both in one step:
    //   down chain: A_p     = Rinv_p     (b_s - C_s y(last)),   s = r1      (separator below)
    //   up chain:   B_{p-1} = -Rinv_{p-1} C_{s'+1} y(first),     s' = r0 - 1 (separator above)
    if (Q > 0) {
        C* parts = reinterpret_cast<C*>(A.parts);
        for (int o = tid; o < nb * W; o += blockDim.x) {
            const int c = o % W, b = o / W;
            if (has_below)
                vin_d[b * 64 + c] = csub(rhs_entry<C>(A, r1, c, b0 + b),
                                         cmul(cmul(csx[c], ccy[r1 - r0]), zr(r1 - 1)[b * W + c]));
            if (has_above) vin_u[b * 64 + c] = cneg(cmul(cmul(csx[c], ccy[0]), zr(r0)[b * W + c]));
        }
        __syncthreads();
        const C* SA = has_below ? consume() : nullptr;
        const C* SB = has_above ? consume() : nullptr;
        if (compute)
            dual_dispatch<C, NJ, BT>(has_below, has_above, SA + lofs, vin_d + vofs, SB + lofs, vin_u + vofs, nb,
                                     vd, vu);
#pragma unroll
        for (int b = 0; b < BT; ++b)
            if (b < nb && rowok && (b & 3) == g) {
                if (has_below) parts[((((int64_t)(b0 + b) * Q + p) * kParts + 0) * A.Wmax) + row] = vd[b];
                if (has_above) parts[((((int64_t)(b0 + b) * Q + p - 1) * kParts + 1) * A.Wmax) + row] = vu[b];
            }
        if (!finish()) return;
    }
    if (Q == 0) return;
    // ---- arrival: the last chunk CTA of group gi (chunks gq0..gq1) solves its separators
    const int NG = A.g.G;
    int* cnt = A.counters + (int64_t)tile * (NG + 1);
    const int gi = p == Q ? NG - 1 : (A.g.sepmap[p] >= 0 ? A.g.sepmap[p] : -A.g.sepmap[p] - 1);
    const int q0 = A.g.gq0[gi], q1 = A.g.gq1[gi], n1 = q1 - q0;
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const bool last = atomicAdd(&cnt[gi], 1) == n1;
        if (last) cnt[gi] = 0;
        flags[0] = last ? 1 : 0;
    }
    __syncthreads();
    if (!flags[0]) return;
    __threadfence();
    C* parts = reinterpret_cast<C*>(A.parts);
    auto pidx = [&](int b, int q, int k) -> int64_t { return (((int64_t)(b0 + b) * Q + q) * kParts + k) * A.Wmax; };
    auto zq = [&](int i) -> C* { return zb + i * BT * W; };
    // one separator step: out_i = z_i - product, stored to z_i and to the chain's next input
    auto sep = [&](auto Dc, auto Uc, int qd, int qu) -> bool {
        constexpr bool D = decltype(Dc)::value, U = decltype(Uc)::value;
        const C* Sd = D ? consume() : nullptr;
        const C* Su = U ? consume() : nullptr;
        if (compute) dual_rows<C, NJ, BT, D, U>(Sd + lofs, vin_d + vofs, Su + lofs, vin_u + vofs, nb, vd, vu);
#pragma unroll
        for (int b = 0; b < BT; ++b)
            if (owns(b)) {
                if (D) {
                    C* zp = zq(qd) + b * W + row;
                    const C x = csub(*zp, vd[b]);
                    *zp = x;
                    vout_d[b * 64 + row] = x;
                }
                if (U) {
                    C* zp = zq(qu) + b * W + row;
                    const C x = csub(*zp, vu[b]);
                    *zp = x;
                    vout_u[b * 64 + row] = x;
                }
            }
        return finish();
    };
    // Twisted solve of n separators whose factors sit at slot(i) (level 1: q0 + i;
    // level 2: gq1[i]); a_i is in zq(i), a_0 / a_{n-1} in vin_d / vin_u.  xe0 / xe1
    // (encoded, or -1) are extra loads appended to the sequence.  Every earlier
    // load has been consumed, so the ring continues from slot cslot.
    auto chain = [&](int n, int lvl, int xe0, int xe1) -> bool {
        const int tq = (n - 1) / 2;
        const int fd = imax(tq - 1, 0), fu = imax(n - 2 - tq, 0), fmx = imax(fd, fu);   // forward steps
        const int bd = tq, bu = n - 1 - tq, bmx = imax(bd, bu);                         // back steps
        sep_phase = true;
        if (producer) {
            auto slot = [&](int i) { return lvl == 1 ? q0 + i : A.g.gq1[i]; };
            int nr = 0;
            for (int s = 0; s < fmx; ++s) {
                if (s < fd) order[nr++] = enc(kEo, slot(1 + s));
                if (s < fu) order[nr++] = enc(kEo, slot(n - 2 - s));
            }
            if (tq >= 1) order[nr++] = enc(kEo, slot(tq));
            if (tq <= n - 2) order[nr++] = enc(kFi, slot(tq));
            for (int s = 0; s < bmx; ++s) {
                if (s < bd) order[nr++] = enc(kFi, slot(tq - 1 - s));
                if (s < bu) order[nr++] = enc(kFi, slot(tq + 1 + s));
            }
            if (xe0 >= 0) order[nr++] = xe0;
            if (xe1 >= 0) order[nr++] = xe1;
            seqbase = consumed;
            nseq = seqbase + nr;
            rf = seqbase;
            rfslot = cslot;
            int sl = cslot;
            for (int i = 0; i < imin(ring, nr); ++i) {
                issue_into(sl, src_of(seqbase + i));
                if (++sl == ring) sl = 0;
            }
        }
        // forward: z_i = a_i - E_i z_outer, down i = 1..tq-1, up i = n-2..tq+1
        {
            int s = 0;
            const int nboth = imin(fd, fu);
            for (; s < nboth; ++s)
                if (!sep(std::true_type{}, std::true_type{}, 1 + s, n - 2 - s)) return false;
            for (; s < fd; ++s)
                if (!sep(std::true_type{}, std::false_type{}, 1 + s, 0)) return false;
            for (; s < fu; ++s)
                if (!sep(std::false_type{}, std::true_type{}, 0, n - 2 - s)) return false;
        }
        // twist: x_tq = a_tq - E_tq z_{tq-1} - F_tq z_{tq+1}
        for (int o = tid; o < nb * W; o += blockDim.x) {
            const int c = o % W, b = o / W;
            if (tq >= 1) vin_d[b * 64 + c] = zq(tq - 1)[b * W + c];
            if (tq <= n - 2) vin_u[b * 64 + c] = zq(tq + 1)[b * W + c];
        }
        __syncthreads();
        {
            const bool he = tq >= 1, hf = tq <= n - 2;
            const C* Se = he ? consume() : nullptr;
            const C* Sf = hf ? consume() : nullptr;
            if (compute)
                dual_dispatch<C, NJ, BT>(he, hf, Se + lofs, vin_d + vofs, Sf + lofs, vin_u + vofs, nb, vd, vu);
#pragma unroll
            for (int b = 0; b < BT; ++b)
                if (b < nb && rowok && (b & 3) == g) {
                    C* zp = zq(tq) + b * W + row;
                    C x = *zp;
                    if (he) x = csub(x, vd[b]);
                    if (hf) x = csub(x, vu[b]);
                    *zp = x;
                    vout_d[b * 64 + row] = x;
                    vout_u[b * 64 + row] = x;
                }
            if (!finish()) return false;
        }
        // back: x_i = z_i - F_i x_inner, down i = tq-1..0, up i = tq+1..n-1
        {
            int s = 0;
            const int nboth = imin(bd, bu);
            for (; s < nboth; ++s)
                if (!sep(std::true_type{}, std::true_type{}, tq - 1 - s, tq + 1 + s)) return false;
            for (; s < bd; ++s)
                if (!sep(std::true_type{}, std::false_type{}, tq - 1 - s, 0)) return false;
            for (; s < bu; ++s)
                if (!sep(std::false_type{}, std::true_type{}, 0, tq + 1 + s)) return false;
        }
        return true;
    };
    // ---- level 1: a_q = A_q + B_q for the group's separators q0 .. q1-1
    const bool up2 = gi > 0, dn2 = gi < NG - 1;   // level-2 separators above / below the group
    for (int o = tid; o < n1 * nb * W; o += blockDim.x) {
        const int c = o % W, b = (o / W) % nb, i = o / (W * nb);
        const int64_t pb = pidx(b, q0 + i, 0) + c;
        const C v = cadd(__ldcg(parts + pb), __ldcg(parts + pb + A.Wmax));
        zb[(i * BT + b) * W + c] = v;
        if (i == 0) vin_d[b * 64 + c] = v;
        if (i == n1 - 1) vin_u[b * 64 + c] = v;
    }
    __syncthreads();
    if (!chain(n1, 1, dn2 ? enc(kP2L, q1) : -1, up2 ? enc(kP2U, q0 - 1) : -1)) return;
    for (int o = tid; o < n1 * nb * W; o += blockDim.x) {
        const int c = o % W, b = (o / W) % nb, i = o / (W * nb);
        yrow<C>(A, b0 + b, A.g.r1[q0 + i])[c] = zb[(i * BT + b) * W + c];
    }
    if (NG == 1) return;
    // ---- the group's parts of the level-2 right-hand sides:
    //   -P2L_{gi} y(last) to the separator below, -P2U_{gi-1} y(first) to the one above
    for (int o = tid; o < nb * W; o += blockDim.x) {
        const int c = o % W, b = o / W;
        if (dn2) vin_d[b * 64 + c] = zq(n1 - 1)[b * W + c];
        if (up2) vin_u[b * 64 + c] = zq(0)[b * W + c];
    }
    __syncthreads();
    {
        const C* SL = dn2 ? consume() : nullptr;
        const C* SU = up2 ? consume() : nullptr;
        if (compute) dual_dispatch<C, NJ, BT>(dn2, up2, SL + lofs, vin_d + vofs, SU + lofs, vin_u + vofs, nb, vd, vu);
#pragma unroll
        for (int b = 0; b < BT; ++b)
            if (b < nb && rowok && (b & 3) == g) {
                if (dn2) parts[pidx(b, q1, 2) + row] = cneg(vd[b]);
                if (up2) parts[pidx(b, q0 - 1, 3) + row] = cneg(vu[b]);
            }
        if (!finish()) return;
    }
    // ---- arrival: the last group to finish solves the level-2 system
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const bool last = atomicAdd(&cnt[NG], 1) == NG - 1;
        if (last) cnt[NG] = 0;
        flags[0] = last ? 1 : 0;
    }
    __syncthreads();
    if (!flags[0]) return;
    __threadfence();
    const int n2 = NG - 1;
    for (int o = tid; o < n2 * nb * W; o += blockDim.x) {
        const int c = o % W, b = (o / W) % nb, i = o / (W * nb);
        const int64_t pb = pidx(b, A.g.gq1[i], 0) + c;
        C v = cadd(__ldcg(parts + pb), __ldcg(parts + pb + A.Wmax));
        v = cadd(v, cadd(__ldcg(parts + pb + 2 * A.Wmax), __ldcg(parts + pb + 3 * A.Wmax)));
        zb[(i * BT + b) * W + c] = v;
        if (i == 0) vin_d[b * 64 + c] = v;
        if (i == n2 - 1) vin_u[b * 64 + c] = v;
    }
    __syncthreads();
    if (!chain(n2, 2, -1, -1)) return;
    for (int o = tid; o < n2 * nb * W; o += blockDim.x) {
        const int c = o % W, b = (o / W) % nb, i = o / (W * nb);
        yrow<C>(A, b0 + b, A.g.r1[A.g.gq1[i]])[c] = zb[(i * BT + b) * W + c];
    }
}

// ------------------------------------------------------------------ spike corrections
// Dot products of spike rows with separator values, 8 lanes per output entry:
// lane g of a group holds the separator entries a = g + 8 i (W <= 64, so i < 8)
// in registers, loads its spike entries with one unrolled batch of independent
// loads, and a three-level butterfly finishes the sum on all 8 lanes.
template <typename C>
__device__ __forceinline__ void lane_vec(C (&v)[8], const C* x, bool on, int g, int W) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int a = g + 8 * i;
        v[i] = (on && a < W) ? x[a] : CT<C>::zero();
    }
}
template <typename C>
__device__ __forceinline__ C spike_dot2(const C* __restrict__ ra, const C (&xa)[8], bool ua,
                                        const C* __restrict__ rb, const C (&xb)[8], bool ub, int g, int W) {
    C sa[8], sb[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int a = g + 8 * i;
        sa[i] = (ua && a < W) ? ra[a] : CT<C>::zero();
        sb[i] = (ub && a < W) ? rb[a] : CT<C>::zero();
    }
    C s0 = CT<C>::zero(), s1 = CT<C>::zero();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        s0 = cfma(sa[i], xa[i], s0);
        s1 = cfma(sb[i], xb[i], s1);
    }
    C s = cadd(s0, s1);
#pragma unroll
    for (int o = 1; o <= 4; o <<= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
    }
    return s;
}

// One CTA per (separator, RHS tile): the grouped separator q of group gi gets
// x_q = y_q - GT2_q x2_{gi-1} - GB2_q x2_{gi} (row-major spikes); level-2
// separators are already final.
template <typename C>
__global__ void __launch_bounds__(512) k_sweep_sepfix(SweepArgs A, const C* __restrict__ GT2,
                                                      const C* __restrict__ GB2) {
    const int q = blockIdx.x;
    const int gi = A.g.sepmap[q];
    if (gi < 0) return;
    const int b0 = blockIdx.y * A.Bt;
    const int nb = imin(A.Bt, A.B - b0);
    const int W = A.st.W;
    const int64_t off = A.st.red + (int64_t)q * A.st.bs;
    const bool up = gi > 0, dn = gi < A.g.G - 1;
    const int ra = up ? A.g.r1[A.g.gq0[gi] - 1] : 0;
    const int rb = dn ? A.g.r1[A.g.gq1[gi]] : 0;
    const int tid = threadIdx.x, g = tid & 7;
    const int c = tid >> 3;                       // the block has 8 lanes per column, W <= 64
    const bool live = c < W;
    const int cc = imin(c, W - 1);
    for (int b = 0; b < nb; ++b) {
        C xa[8], xb[8];
        lane_vec(xa, yrow<C>(A, b0 + b, ra), up, g, W);
        lane_vec(xb, yrow<C>(A, b0 + b, rb), dn, g, W);
        const C s = spike_dot2(GT2 + off + (int64_t)cc * W, xa, up, GB2 + off + (int64_t)cc * W, xb, dn, g, W);
        if (live && g == 0) {
            C* y = yrow<C>(A, b0 + b, A.g.r1[q]);
            y[c] = csub(y[c], s);
        }
    }
}

// One CTA per (row, RHS tile): x_k = y_k - GT_p(k) x_{p-1} - GB_p(k) x_p on the
// output columns and the two transfer columns; the owning lane scatters x
// (plus the base field) to the output, and the transfer difference is emitted.
template <typename C>
__global__ void __launch_bounds__(256) k_sweep_correct(SweepArgs A, const C* __restrict__ GT,
                                                       const C* __restrict__ GB) {
    const int k = blockIdx.x;
    const int b0 = blockIdx.y * A.Bt;
    const int nb = imin(A.Bt, A.B - b0);
    const int W = A.st.W;
    const int64_t bs = A.st.bs;
    __shared__ C xt[8];   // the two transfer columns, per RHS (Bt <= 4)
    const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
    const int pm = A.g.rowmap[k];
    const int off = A.st.lo - A.st.lpml;
    const int olo = imax(A.sp.olo - off, 0), ohi = imin(A.sp.ohi - off, W - 1);
    const int nout = imax(ohi - olo + 1, 0);
    const bool tr = A.sp.tout != nullptr;
    const bool x0 = tr && (A.sp.to0 < olo || A.sp.to0 > ohi);
    const bool x1 = tr && (A.sp.to1 < olo || A.sp.to1 > ohi);
    const int ncol = nout + (x0 ? 1 : 0) + (x1 ? 1 : 0);
    const bool above = pm > 0, below = pm >= 0 && pm < A.g.P - 1;
    const int g = l & 7;
    const int64_t rowoff = A.st.fac + (int64_t)k * bs;
    for (int b = 0; b < nb; ++b) {
        C xa[8], xb[8];
        lane_vec(xa, yrow<C>(A, b0 + b, above ? A.g.r1[pm - 1] : 0), above, g, W);
        lane_vec(xb, yrow<C>(A, b0 + b, below ? A.g.r1[pm] : 0), below, g, W);
        for (int base = w * 4; base < ncol; base += (blockDim.x >> 5) * 4) {   // warp-uniform trip count
            // column i of this 8-lane group; groups past ncol idle but join the shuffles
            const int i = base + (l >> 3);
            const bool live = i < ncol;
            int c = olo;
            if (live) {
                if (i < nout) c = olo + i;
                else if (i == nout && x0) c = A.sp.to0;
                else c = A.sp.to1;
            }
            const int cs = imin(imax(c, 0), W - 1);
            const C s = spike_dot2(GT + rowoff + (int64_t)cs * W, xa, above, GB + rowoff + (int64_t)cs * W, xb,
                                   below, g, W);
            if (live && g == 0) {
                const C x = csub(yrow<C>(A, b0 + b, k)[c], s);
                const int64_t rowi = (int64_t)(b0 + b) * A.g.Ny + k;
                if (c >= olo && c <= ohi) {
                    double2 v = to_d2(x);
                    if (A.sp.base) v = cadd(v, A.sp.base[rowi * A.g.Nx + off + c]);
                    A.sp.dst[rowi * A.g.Nx + off + c] = v;
                }
                if (tr && c == A.sp.to0) xt[b * 2] = x;
                if (tr && c == A.sp.to1) xt[b * 2 + 1] = x;
            }
        }
    }
    if (!tr) return;
    __syncthreads();
    for (int b = tid; b < nb; b += blockDim.x)
        A.sp.tout[(int64_t)(b0 + b) * A.g.Ny + k] = csub(to_d2(xt[b * 2 + 1]), to_d2(xt[b * 2]));
}

// ------------------------------------------------------------------ host
template <typename C>
static SweepArgs make_args(const Geom& g, const StripDev& st, const SweepStep& step, const SweepWork& wk,
                           void* const* pool, int Bt, int ring) {
    SweepArgs A;
    A.g = g;
    A.st = st;
    A.sp = step;
    A.Wmax = wk.Wmax;
    A.B = wk.B;
    A.Bt = Bt;
    A.ring = ring;
    A.zrows = wk.zrows;
    A.slot_bytes = (uint32_t)(st.bs * sizeof(C));
    A.Sinv = pool[0];
    A.Rinv = pool[3];
    A.E = pool[4];
    A.F = pool[5];
    A.P2L = g.G > 1 ? pool[8] : nullptr;
    A.P2U = g.G > 1 ? pool[9] : nullptr;
    A.ybuf = wk.ybuf;
    A.parts = wk.parts;
    A.counters = wk.counters;
    A.status = wk.status;
    return A;
}

// Largest ring (and RHS tile) that fits the shared-memory budget.
template <typename C>
static bool plan(const StripDev& st, int zrows, int B, int& Bt, int& ring, size_t& smem) {
    const size_t budget = 220 * 1024;
    const uint32_t slot = (uint32_t)(st.bs * sizeof(C));
    for (Bt = (B > 1 ? 4 : 1); Bt >= 1; Bt -= 3) {   // tiles of 4 right-hand sides, or 1
        for (ring = kMaxRing; ring >= 4; --ring) {
            smem = sweep_smem(ring, slot, zrows, Bt, st.W, (int)sizeof(C)).total;
            if (smem <= budget) return true;
        }
    }
    return false;
}

template <typename C>
cudaError_t launch_strip_solve(const Geom& g, int j, const StripDev& st, const SweepStep& step,
                               const SweepWork& wk, void* const* pool, cudaStream_t s, KernelTimer* tm) {
    int Bt, ring;
    size_t smem;
    if (!plan<C>(st, wk.zrows, wk.B, Bt, ring, smem)) return cudaErrorInvalidConfiguration;
    static bool attr_set = false;
    if (!attr_set) {
        for (auto fn : {k_sweep_chunk<C, 8, 1>, k_sweep_chunk<C, 10, 1>, k_sweep_chunk<C, 12, 1>,
                        k_sweep_chunk<C, 14, 1>, k_sweep_chunk<C, 16, 1>, k_sweep_chunk<C, 8, 4>,
                        k_sweep_chunk<C, 10, 4>, k_sweep_chunk<C, 12, 4>, k_sweep_chunk<C, 14, 4>,
                        k_sweep_chunk<C, 16, 4>}) {
            cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
            if (e != cudaSuccess) return e;
        }
        attr_set = true;
    }
    SweepArgs A = make_args<C>(g, st, step, wk, pool, Bt, ring);
    const int ntile = (wk.B + Bt - 1) / Bt;
    {
        TimedLaunch t(tm, "sweep_chunk", s);
        const dim3 grid(g.P, ntile);
        const int nthr = 32 * ((st.W + 7) / 8 + 1);   // compute warps + the producer warp
#define HELM_LAUNCH_CHUNK(NJ)                                                         \
    (Bt == 1 ? (k_sweep_chunk<C, NJ, 1><<<grid, nthr, smem, s>>>(A), 0)              \
             : (k_sweep_chunk<C, NJ, 4><<<grid, nthr, smem, s>>>(A), 0))
        switch (st.nj) {
            case 8: HELM_LAUNCH_CHUNK(8); break;
            case 10: HELM_LAUNCH_CHUNK(10); break;
            case 12: HELM_LAUNCH_CHUNK(12); break;
            case 14: HELM_LAUNCH_CHUNK(14); break;
            default: HELM_LAUNCH_CHUNK(16); break;
        }
#undef HELM_LAUNCH_CHUNK
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    if (g.G > 1) {
        TimedLaunch t(tm, "sweep_sepfix", s);
        k_sweep_sepfix<C><<<dim3(g.P - 1, ntile), 8 * ((st.W + 3) & ~3), 0, s>>>(A, (const C*)pool[6],
                                                                                (const C*)pool[7]);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    {
        TimedLaunch t(tm, "sweep_correct", s);
        // one warp per output column (the strip's output range plus the transfer columns)
        const int ncol = (step.ohi - step.olo + 1) + 2;
        const int nthr = 32 * imin(8, imax(1, (ncol + 3) / 4));
        k_sweep_correct<C><<<dim3(g.Ny, ntile), nthr, 0, s>>>(A, (const C*)pool[1], (const C*)pool[2]);
    }
    return cudaGetLastError();
}

template cudaError_t launch_strip_solve<float2>(const Geom&, int, const StripDev&, const SweepStep&,
                                                const SweepWork&, void* const*, cudaStream_t, KernelTimer*);
template cudaError_t launch_strip_solve<double2>(const Geom&, int, const StripDev&, const SweepStep&,
                                                 const SweepWork&, void* const*, cudaStream_t, KernelTimer*);

}  // namespace helm
