// One strip solve of the double sweep (Section 2.1, Eqs. solve_upward and
// solve_downward) on the partitioned block-tridiagonal factors of factor.cu.
//
// k_sweep_chunk (grid: chunks x RHS tiles)
//   * builds the strip right-hand side S^(j) r for every row of its chunk
//     (masked source plus the single-layer-potential transfer on two columns,
//     which it takes directly from the previous strip solve's chain and group
//     solutions through the transfer composites of factor.cu);
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
// k_sweep_output (work items: chunks x strips x RHS tiles, grid-stride)
//   final separator values (grouped separators: x_q = y_q - GT2_q x2_above -
//   GB2_q x2_below), then x_k = y_k - GT_p(k) x_{p-1} - GB_p(k) x_p on the output
//   columns of every strip, scattered (plus the base field) to the output field.
//
// Every mbarrier wait is bounded; on time-out the kernel records
// HELM_ETIMEOUT in the status word, drains its copies (bounded) and returns.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace helm {

static constexpr int kMaxRing = 32;
static constexpr uint32_t kWaitLimit = 1u << 22;
static constexpr int kParts = 2;   // separator right-hand-side parts, one from each neighbouring chunk
static constexpr int kAhead = 6;   // block loads in flight ahead of the chain (three dual steps)

// load-order table entries: factor pool << 24 | block index in that pool
enum : int { kSinv = 0, kRinv = 1, kEo = 2, kFi = 3, kQ2L = 4, kQ2U = 5 };
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
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
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
// Programmatic dependent launch: the chunk and transfer kernels of consecutive
// strip solves are launched with programmatic stream serialisation.  A kernel
// lets its successor's CTAs be scheduled at once (launch_dependents) and does
// its own independent set-up (barriers, staging factor blocks, tables) before
// waiting for its predecessor to complete and flush (wait); everything it
// reads or writes that a predecessor touches comes after that wait.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

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
    const void* Q2L;         // level-2 contributions of a group separator's part (null with one group)
    const void* Q2U;
    void* ybuf;              // [B][Ny][Wmax] chunk solutions, then separator values
    void* parts;             // [B][P-1][kParts][Wmax] separator right-hand-side parts
    void* acc2;              // [B][G-1][Wmax] the level-2 right-hand sides' shares from the group
                             // separators, summed by the chunks' atomic adds; zero between launches
    // the previous strip solve, whose transfer enters this one (has_prev)
    int has_prev;
    StripDev pst;
    const void* pybuf;       // its chain solution [B][Ny][Wmax]
    const void* GT;          // spike pools (all strips)
    const void* GB;
    const void* GT2;
    const void* GB2;
    const void* XF;          // transfer composites (with separator groups)
    int* counters;           // [ntile][G+1] arrival counters, left at zero
    int* status;
};

template <typename C>
__device__ __forceinline__ const C* ctab(const Geom& g) { return reinterpret_cast<const C*>(g.ct); }

template <typename C>
__device__ __forceinline__ C coupling(const SweepArgs& A, int k, int c) {
    return cmul(ctab<C>(A.g)[A.st.ctab + c], ctab<C>(A.g)[A.g.ct_cy + k]);
}

template <typename C>
__device__ __forceinline__ C* yrow(const SweepArgs& A, int b, int k) {
    return reinterpret_cast<C*>(A.ybuf) + ((int64_t)b * A.g.Ny + k) * A.Wmax;
}

// Shared-memory carve-up (bytes), identical on host and device.
struct SweepSmem {
    uint32_t slots, zb, tv, cx, cy, xv, order, l2, mbar, flags, total;
};
__host__ __device__ inline SweepSmem sweep_smem(int ring, uint32_t slot_bytes, int zrows, int Bt, int W,
                                                int esz) {
    SweepSmem s;
    uint32_t o = 0;
    s.slots = o; o += ring * slot_bytes;
    s.zb = o; o += ((uint32_t)zrows * Bt * W * esz + 15u) & ~15u;
    s.tv = o; o += 8u * Bt * 64 * esz;        // in/out vectors of both chains, separator-row rhs, parts inputs, zero
    s.cx = o; o += 64u * esz;
    s.cy = o; o += ((uint32_t)(zrows + 2) * esz + 15u) & ~15u;
    s.xv = o; o += ((uint32_t)(6 * Bt * 64 + (zrows + 1) * Bt * 2) * esz + 15u) & ~15u;   // incoming transfer
    s.order = o; o += ((uint32_t)(6 * zrows + 8) * 4 + 15u) & ~15u;   // load order table
    s.l2 = o; o += 64 * 4;                                               // level-2 separators (first 64)
    s.mbar = o; o += kMaxRing * 8;
    s.flags = o; o += 16;
    s.total = o;
    return s;
}

// Load order of a twisted separator chain over n elements (consumed in the
// same order by `chain` in k_sweep_chunk): the forward E loads of both halves
// interleaved, E and F of the twist, then the back F loads.  slot(i) is the
// factor slot of element i.
template <typename SL>
__device__ int chain_order(int* ord, int n, SL slot) {
    const int tq = (n - 1) / 2;
    const int fd = imax(tq - 1, 0), fu = imax(n - 2 - tq, 0), fmx = imax(fd, fu);
    const int bd = tq, bu = n - 1 - tq, bmx = imax(bd, bu);
    int nr = 0;
    for (int s = 0; s < fmx; ++s) {
        if (s < fd) ord[nr++] = enc(kEo, slot(1 + s));
        if (s < fu) ord[nr++] = enc(kEo, slot(n - 2 - s));
    }
    if (tq >= 1) ord[nr++] = enc(kEo, slot(tq));
    if (tq <= n - 2) ord[nr++] = enc(kFi, slot(tq));
    for (int s = 0; s < bmx; ++s) {
        if (s < bd) ord[nr++] = enc(kFi, slot(tq - 1 - s));
        if (s < bu) ord[nr++] = enc(kFi, slot(tq + 1 + s));
    }
    return nr;
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
// The factor rows sd, su are already in registers (loaded from the blocks' shared-memory
// slots, possibly during the previous step).
template <typename C, int NJ, int BT, bool D, bool U>
__device__ __forceinline__ void dual_rows_r(const C (&sd)[NJ], const C (&su)[NJ], const C* __restrict__ td,
                                            const C* __restrict__ tu, int nb, C (&vd)[BT], C (&vu)[BT]) {
#pragma unroll
    for (int b = 0; b < BT; ++b) {
        if (BT == 1 || b < nb) {   // nb >= 1: no test for a single right-hand side
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

// The CTA is ceil(W/8) compute warps plus one producer warp.  The producer's
// lane 0 owns the TMA ring: it initialises the barriers, issues every bulk
// copy, and right after each step's barrier refills the slots that step
// consumed, while the compute warps already run the next step.  All factor
// blocks the CTA may need form one load sequence: the chunk's Sinv rows and
// the two Rinv blocks, then the chain of the chunk's separator group and the
// level-2 chain.  Every CTA streams the start of the separator chains into
// its free slots while it finishes the chunk; the CTA that arrives last at
// its group solves the group with those blocks already resident, the others
// wait for their copies to land and exit.
template <typename C, int NJ, int BT>
__global__ void __launch_bounds__(288) k_sweep_chunk(SweepArgs A) {
    using R = typename CT<C>::R;
    extern __shared__ __align__(128) unsigned char smem[];
    pdl_trigger();
    constexpr int LD = 4 * NJ + 2;
    const int W = A.st.W;
    const int esz = (int)sizeof(C);
    const SweepSmem L = sweep_smem(A.ring, A.slot_bytes, A.zrows, BT, W, esz);
    unsigned char* slots = smem + L.slots;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L.mbar);
    C* zb = reinterpret_cast<C*>(smem + L.zb);       // [zrows][BT][W]
    C* xv = reinterpret_cast<C*>(smem + L.xv);       // incoming transfer: [6][BT][64] vectors, [rows][BT][2] values
    C* v0 = reinterpret_cast<C*>(smem + L.tv);       // [BT][64] vectors: in/out of both chains, separator rhs
    C* vin_d = v0;
    C* vin_u = v0 + BT * 64;
    C* vout_d = v0 + 2 * BT * 64;
    C* vout_u = v0 + 3 * BT * 64;
    C* rsep = v0 + 4 * BT * 64;                      // S r on the separator row below the chunk
    // inputs of the steps after a chain (separator right-hand-side parts), written by
    // the owner lanes of each half's last step: pv_d from the down half, pv_u from the up half
    C* pv_d = v0 + 5 * BT * 64;
    C* pv_u = v0 + 6 * BT * 64;
    const C* vzero = v0 + 7 * BT * 64;               // stays zero
    C* csx = reinterpret_cast<C*>(smem + L.cx);      // s_x(c)
    C* ccy = reinterpret_cast<C*>(smem + L.cy);      // -alpha_y(k-1/2)/h^2, k = r0..r1
    int* order = reinterpret_cast<int*>(smem + L.order);
    int* l2s = reinterpret_cast<int*>(smem + L.l2);  // level-2 separator indices gq1[i], i < 64
    volatile int* flags = reinterpret_cast<int*>(smem + L.flags);
    const int p = blockIdx.x, tile = blockIdx.y;
    // with separator groups one more CTA (p = P) solves the level-2 system: it starts once
    // every chunk has added its contributions to the level-2 right-hand sides, while the
    // last chunk of each group solves the group
    const bool l2cta = A.g.G > 1 && p == A.g.P;
    const int pc = l2cta ? 0 : p;                    // geometry lookups of the level-2 CTA stay in range
    const int b0 = tile * BT;
    const int nb = imin(BT, A.B - b0);
    const int r0 = A.g.r0[pc], r1 = A.g.r1[pc], m = r1 - r0;
    const int t = r0 + (m - 1) / 2;                  // twist row
    const int nd = t - r0, nu = r1 - 1 - t, nmx = imax(nd, nu);
    const int P = A.g.P, Q = P - 1;
    const int tid = threadIdx.x;
    const int ptid = blockDim.x - 32;                // the producer warp starts here; threads below compute
    const bool producer = tid == ptid;               // its lane 0: barriers, order table, status
    const bool pwarp = tid >= ptid;                  // all its lanes issue copies, one each
    const int plane = tid - ptid;
    const bool compute = tid < ptid;
    const int64_t bs = A.st.bs;
    const int ring = A.ring;
    const uint32_t sb = A.slot_bytes;
    const C* Sinv = reinterpret_cast<const C*>(A.Sinv) + A.st.fac;
    const C* Rinv = reinterpret_cast<const C*>(A.Rinv) + A.st.red;
    const C* Eb = reinterpret_cast<const C*>(A.E) + A.st.red;
    const C* Fb = reinterpret_cast<const C*>(A.F) + A.st.red;
    const C* Q2Lb = A.Q2L ? reinterpret_cast<const C*>(A.Q2L) + A.st.red : nullptr;
    const C* Q2Ub = A.Q2U ? reinterpret_cast<const C*>(A.Q2U) + A.st.red : nullptr;
    const bool resident = ring >= m + 2;
    const bool has_below = !l2cta && p < P - 1, has_above = !l2cta && p > 0;
    // separator group of this chunk: group gi owns separators gq0..gq1-1 and chunks gq0..gq1
    const int NG = A.g.G;
    const int gi = Q == 0 ? 0 : (pc == Q ? NG - 1 : (A.g.sepmap[pc] >= 0 ? A.g.sepmap[pc] : -A.g.sepmap[pc] - 1));
    const int q0 = Q == 0 ? 0 : A.g.gq0[gi], q1 = Q == 0 ? 0 : A.g.gq1[gi], n1 = q1 - q0;
    const int n2 = NG - 1;
    // this chunk's contributions to the level-2 right-hand sides: its part of separator p
    // (below) and of separator p-1 (above), each through the contribution block of that
    // separator toward the level-2 separator below (q2dn) or above (q2up) its group
    auto grp_of = [&](int q) { return A.g.sepmap[q]; };   // >= 0: a group member; < 0: a level-2 separator
    const bool q2dnA = NG > 1 && has_below && grp_of(p) >= 0 && grp_of(p) < NG - 1;
    const bool q2dnB = NG > 1 && has_above && grp_of(p - 1) >= 0 && grp_of(p - 1) < NG - 1;
    const bool q2upA = NG > 1 && has_below && grp_of(p) > 0;
    const bool q2upB = NG > 1 && has_above && grp_of(p - 1) > 0;
    // ---- ring state: load G lives in slot G % ring and completes phase (G / ring) & 1
    int nload = 0;                          // producer warp: length of the load sequence
    int cap = 0;                            // producer warp: loads from cap on wait for the next arrival
    int issued = 0, consumed = 0;
    int cslot = 0;
    uint32_t cpar = 0;
    bool hold = resident && !l2cta;         // a resident chunk's slots are read again by the back pass
    int nchunk = 0, ngroup = 0;             // producer warp: loads of the chunk and of the group chain
    auto src_of = [&](int G) -> const C* {
        const int e = order[G];
        const int64_t o = (int64_t)(e & 0xffffff) * bs;
        switch (e >> 24) {
            case kSinv: return Sinv + o;
            case kRinv: return Rinv + o;
            case kEo: return Eb + o;
            case kFi: return Fb + o;
            case kQ2L: return Q2Lb + o;
            default: return Q2Ub + o;
        }
    };
    // producer warp: issue loads issued .. lim-1 (at most one ring, one per lane) together
    auto issue_upto = [&](int lim) {
        const int n = lim - issued;
        if (n <= 0) return;
        if (plane < n) {
            const int G = issued + plane, slot = G % ring;
            uint64_t* mb = &mbar[slot];
            fence_proxy_async();
            mbar_expect_tx(mb, sb);
            bulk_g2s(slots + (size_t)slot * sb, src_of(G), sb, mb);
        }
        issued = lim;
    };
    bool late = false;   // this thread's bounded wait gave up (reduced over the CTA in finish)
    auto consume = [&]() -> const C* {
        const C* S = reinterpret_cast<const C*>(slots + (size_t)cslot * sb);
        if (compute && !mbar_wait(&mbar[cslot], cpar)) late = true;
        ++consumed;
        if (++cslot == ring) { cslot = 0; cpar ^= 1u; }
        return S;
    };
    // the next one or two loads of the sequence, their barriers polled together
    auto consume2 = [&](bool two, const C*& S1, const C*& S2) {
        const int s1 = cslot;
        const uint32_t p1 = cpar;
        int s2 = cslot + 1;
        uint32_t p2 = cpar;
        if (s2 == ring) { s2 = 0; p2 ^= 1u; }
        S1 = reinterpret_cast<const C*>(slots + (size_t)s1 * sb);
        S2 = two ? reinterpret_cast<const C*>(slots + (size_t)s2 * sb) : S1;
        if (compute) {
            bool ok1 = false, ok2 = !two;
            for (uint32_t it = 0; it < kWaitLimit && !(ok1 && ok2); ++it) {
                if (!ok1) ok1 = mbar_try_wait(&mbar[s1], p1);
                if (!ok2) ok2 = mbar_try_wait(&mbar[s2], p2);
            }
            if (!(ok1 && ok2)) late = true;
        }
        const int k = two ? 2 : 1;
        consumed += k;
        cslot += k;
        if (cslot >= ring) { cslot -= ring; cpar ^= 1u; }
    };
    // producer warp, after a barrier: keep kAhead loads in flight, each into a
    // slot whose previous load has been consumed (and is no longer held)
    auto refill = [&]() {
        const int room = hold ? ring : consumed + ring;
        // the level-2 CTA fills its whole ring while it waits for the chunks
        issue_upto(imin(imin(cap, nload), imin(room, consumed + (l2cta ? ring : kAhead))));
    };
    // producer: wait (bounded) for the copies still in flight from load `from` on
    auto land = [&](int from) {
        if (producer)
            for (int Gd = imax(from, 0); Gd < issued; ++Gd) mbar_wait(&mbar[Gd % ring], (uint32_t)((Gd / ring) & 1));
    };
    auto abort_wait = [&]() {   // a bounded wait gave up: report, let the copies land, leave
        if (producer) atomicExch(A.status, 7);
        land(consumed - 2);   // the step's one or two loads and every later copy
        __syncthreads();
    };
    if (producer) {
        for (int i = 0; i < ring; ++i) mbar_init(&mbar[i], 1);
        fence_mbar_init();
    }
    for (int o = tid; o < 8 * BT * 64; o += blockDim.x) v0[o] = CT<C>::zero();
    __syncthreads();   // barriers initialised, vectors zeroed
    const C* ct = ctab<C>(A.g);
    if (producer && l2cta) {   // the level-2 CTA: the level-2 chain only
        for (int i = 0; i < imin(n2, 64); ++i) l2s[i] = A.g.gq1[i];
        nload = chain_order(order, n2, [&](int i) { return i < 64 ? l2s[i] : A.g.gq1[i]; });
        nchunk = nload;
    } else if (producer) {
        // load order: the chunk's blocks (with the contribution blocks of its two
        // separators), then the group's separator chain, whose slots come from global memory
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
        if (q2dnA) order[G++] = enc(kQ2L, p);
        if (q2dnB) order[G++] = enc(kQ2L, p - 1);
        if (q2upA) order[G++] = enc(kQ2U, p);
        if (q2upB) order[G++] = enc(kQ2U, p - 1);
        nchunk = G;
        if (Q > 0) {
            G += chain_order(order + G, n1, [&](int i) { return q0 + i; });
            ngroup = G - nchunk;
        }
        nload = G;
    }
    if (pwarp) {
        __syncwarp();
        nload = __shfl_sync(0xffffffffu, nload, 0);
        nchunk = __shfl_sync(0xffffffffu, nchunk, 0);
        ngroup = __shfl_sync(0xffffffffu, ngroup, 0);
        // the chunk's blocks and the first two steps of the group's separator chain:
        // only the CTA that solves the group uses those, the others let them land
        cap = nchunk + imin(4, ngroup);
        refill();
        // the group's first chunk stages the group's separator chain in L2 for whichever
        // CTA ends up solving it
        auto stage_l2 = [&](int from, int to) {
            for (int G = from + plane; G < to; G += 32) bulk_prefetch_l2(src_of(G), sb);
        };
        if (!l2cta && Q > 0 && p == q0) stage_l2(nchunk, nchunk + ngroup);
        if (l2cta) stage_l2(ring, nload);   // the level-2 chain's blocks beyond the ring, into L2
        pdl_wait();
    } else if (l2cta) {
        pdl_wait();   // the counters and buffers of the previous strip solve are settled
    } else {
        // tables and the source part of the right-hand sides S^(j) r of the chunk
        // rows and of the separator row below (the source field is complete before
        // the sweep starts), four entries per thread with all their loads in flight;
        // then, once the previous strip solve is done, its transfer on two columns
        for (int c = tid; c < W; c += ptid) csx[c] = ct[A.st.ctab + c];
        for (int k = r0 + tid; k <= r1; k += ptid) ccy[k - r0] = ct[A.g.ct_cy + k];
        const int nrow = m + (has_below ? 1 : 0);
        const int tot = nrow * nb * W;
        const int cofs = A.st.lo - A.st.lpml;
        auto put = [&](int r, int b, int c, const C& v) {   // chain inputs and the separator row
            if (r < m) {
                zb[(r * BT + b) * W + c] = v;
                if (r == 0 && nd > 0) vin_d[b * 64 + c] = v;       // down chain starts at r0
                if (r == m - 1 && nu > 0) vin_u[b * 64 + c] = v;   // up chain starts at r1-1
            } else {
                rsep[b * 64 + c] = v;
            }
        };
        for (int o0 = tid; o0 < tot; o0 += 4 * ptid) {
            double2 sv[4];
            C sx[4], sy[4];
            int cc[4], bb[4], rr[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {   // loads only (clamped indices, no branches)
                const int o = imin(o0 + u * ptid, tot - 1);
                cc[u] = o % W;
                bb[u] = (o / W) % nb;
                rr[u] = o / (W * nb);
                const int64_t rowi = (int64_t)(b0 + bb[u]) * A.g.Ny + r0 + rr[u];
                sv[u] = __ldg(A.sp.src + rowi * A.g.Nx + imin(imax(cofs + cc[u], 0), A.g.Nx - 1));
                sx[u] = ct[A.st.ctab + cc[u]];
                sy[u] = ct[A.g.ct_sy + r0 + rr[u]];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (o0 + u * ptid >= tot) continue;
                const int gc = cofs + cc[u];
                const double2 f = (gc >= A.sp.mlo && gc <= A.sp.mhi) ? sv[u] : make_double2(0.0, 0.0);
                put(rr[u], bb[u], cc[u], cmul(CT<C>::from(f), cmul(sx[u], sy[u])));
            }
        }
        // The previous strip solve's transfer x[to1] - x[to0] on this chunk's rows and the
        // separator row below, from its chain solution y, the group solutions y2 of the
        // chunk's two separators and the level-2 values x2 around their groups (the
        // composites XF of factor.cu):
        //   chunk row k:   x_k = y_k - GT[c,:] y2_{p-1} - GB[c,:] y2_p + XF[k][c] . x2
        //   separator row: x = y2_p - GT2_p[c,:] x2a - GB2_p[c,:] x2b
        // Tasks (row, column) go to 8-lane groups; the six factor rows of a group's first
        // task are read before the dependency wait (they do not depend on it), the six
        // vectors are staged in shared memory after it.
        const StripDev& ps = A.pst;
        const int Wp = ps.W, SLp = spld(Wp);
        const int4 cm0 = A.g.cmeta[2 * p], cm1 = A.g.cmeta[2 * p + 1];
        const int gA = cm0.z, gB = cm0.w;
        const bool fa0 = gA > 0, fa1 = gA >= 0 && gA < NG - 1, fb0 = gB > 0, fb1 = gB >= 0 && gB < NG - 1;
        const int lg = tid & 7, grp = tid >> 3, ngrp = ptid >> 3;
        const int ntask = A.has_prev ? nrow * 2 : 0;
        // the six rows of task t (unused ones zero), and the signs / switches they go with
        const bool on[6] = {has_above, has_below, fa0, fa1, fb0, fb1};
        auto task_rows = [&](int task, C (&rw)[6][8]) {
            const int kk = task >> 1, i = task & 1;
            const int col = 2 * A.sp.pdir + i, c = ps.xc[col];
            const C* rp[6];
            if (kk < m) {
                const int k = r0 + kk;
                const int64_t ro = ps.fac + (int64_t)k * ps.bs + (int64_t)c * SLp;
                const int64_t xo = ps.xf + ((int64_t)k * 4 + col) * 4 * SLp;
                const C* XFp = reinterpret_cast<const C*>(A.XF);
                rp[0] = reinterpret_cast<const C*>(A.GT) + ro;
                rp[1] = reinterpret_cast<const C*>(A.GB) + ro;
                for (int v = 2; v < 6; ++v) rp[v] = NG > 1 ? XFp + xo + (v - 2) * SLp : nullptr;
            } else {   // the separator row below: only its level-2 spikes
                const int64_t o2 = ps.red + (int64_t)p * ps.bs + (int64_t)c * SLp;
                rp[0] = rp[1] = rp[2] = rp[3] = nullptr;
                rp[4] = NG > 1 ? reinterpret_cast<const C*>(A.GT2) + o2 : nullptr;
                rp[5] = NG > 1 ? reinterpret_cast<const C*>(A.GB2) + o2 : nullptr;
            }
#pragma unroll
            for (int v = 0; v < 6; ++v)
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int a = lg + 8 * q;
                    rw[v][q] = (rp[v] && on[v] && a < Wp) ? rp[v][a] : CT<C>::zero();
                }
        };
        C rw0[6][8];
        if (ntask > 0) task_rows(imin(grp, ntask - 1), rw0);
        pdl_wait();
        if (A.has_prev) {
            const C* Yp = reinterpret_cast<const C*>(A.pybuf);
            // vectors: y2 above (row r0-1), y2 below (row r1), x2 around the group above, below
            const int vrow[6] = {r0 - 1, r1, cm1.x, cm1.y, cm1.z, cm1.w};
            for (int o = tid; o < 6 * nb * 64; o += ptid) {   // zero beyond Wp: the products read all 64
                const int v = o / (nb * 64), b = (o / 64) % nb, c = o % 64;
                xv[(v * BT + b) * 64 + c] = (on[v] && c < Wp)
                                                ? Yp[((int64_t)(b0 + b) * A.g.Ny + vrow[v]) * A.Wmax + c]
                                                : CT<C>::zero();
            }
            asm volatile("bar.sync 1, %0;" ::"r"(ptid) : "memory");
            C* xt = xv + 6 * BT * 64;                       // [row][BT][2]
            const R sg[6] = {(R)-1, (R)-1, (R)1, (R)1, (R)1, (R)1};   // signs of the six terms (chunk rows)
            for (int t0 = 0; t0 < ntask; t0 += ngrp) {   // uniform trip count: every lane shuffles
                const bool live = t0 + grp < ntask;
                const int task = imin(t0 + grp, ntask - 1);
                const int kk = task >> 1, i = task & 1;
                const int c = ps.xc[2 * A.sp.pdir + i];
                if (t0 > 0) task_rows(task, rw0);   // the first task's rows were read before the wait
                const bool srow = kk >= m;           // the separator row: x = y2_p - level-2 terms
                for (int b = 0; b < nb; ++b) {
                    const C y = lg == 0 ? (srow ? xv[(1 * BT + b) * 64 + c]
                                                : Yp[((int64_t)(b0 + b) * A.g.Ny + r0 + kk) * A.Wmax + c])
                                        : CT<C>::zero();
                    C acc = CT<C>::zero();
#pragma unroll
                    for (int v = 0; v < 6; ++v) {
                        C d = CT<C>::zero();
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int a = imin(lg + 8 * q, 63);
                            d = cfma(rw0[v][q], xv[(v * BT + b) * 64 + a], d);
                        }
                        acc = cadd(acc, cscale(d, srow ? (R)-1 : sg[v]));
                    }
#pragma unroll
                    for (int o = 1; o <= 4; o <<= 1) {
                        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
                    }
                    if (live && lg == 0) xt[(kk * BT + b) * 2 + i] = cadd(y, acc);
                }
            }
            asm volatile("bar.sync 1, %0;" ::"r"(ptid) : "memory");
            // tcoef (x[to1] - x[to0]) enters this strip on columns t0, t0+1 (Eqs. solve_upward,
            // solve_downward), scaled to the symmetric form like the source; with Robin
            // transmission (Section 4.4) the Robin data enters the one boundary column
            for (int o = tid; o < nrow * nb * 2; o += ptid) {
                const int i = o & 1, b = (o >> 1) % nb, r = (o >> 1) / nb;
                const int c = A.sp.t0 + i - cofs;
                if (c < 0 || c >= W) continue;
                C tv;
                if (A.sp.rbk) {   // Robin data a x_in + b x_out, over b h^2 (tcoef = 1/h^2)
                    const C w = CT<C>::from(A.sp.rbk[r0 + r]);
                    tv = cadd(cmul(w, xt[(r * BT + b) * 2 + A.sp.rb_in]), xt[(r * BT + b) * 2 + 1 - A.sp.rb_in]);
                } else {
                    tv = csub(xt[(r * BT + b) * 2 + 1], xt[(r * BT + b) * 2]);
                }
                const C add = cmul(cscale(tv, (R)A.sp.tcoef), cmul(ct[A.st.ctab + c], ct[A.g.ct_sy + r0 + r]));
                const C* cur = r < m ? &zb[(r * BT + b) * W + c] : &rsep[b * 64 + c];
                put(r, b, c, cadd(*cur, add));
            }
        }
    }
    __syncthreads();
    // per-lane geometry
    const int w = tid >> 5, l = tid & 31;
    const int row = w * 8 + (l >> 2);
    const int g = l & 3;
    const bool rowok = compute && row < W;
    const int rc = imin(row, W - 1);
    const int lofs = rc * LD + g * NJ;     // this lane's run inside a block
    const int vofs = g * NJ;               // ... and inside a vector
    const C csx_r = compute ? csx[rc] : CT<C>::zero();
    auto zr = [&](int k) -> C* { return zb + (k - r0) * BT * W; };   // row k, b = 0
    auto cpl = [&](int k) -> C { return cmul(csx_r, ccy[k - r0]); }; // C_k at this lane's row
    auto finish = [&]() -> bool {
        if (__syncthreads_or(late)) { abort_wait(); return false; }
        if (pwarp) refill();
        C* x = vin_d; vin_d = vout_d; vout_d = x;
        x = vin_u; vin_u = vout_u; vout_u = x;
        return true;
    };
    C vd[BT], vu[BT];
    // The products of a step, vd = Sd-row . td and vu = Su-row . tu, in one
    // instruction stream for both chains.  A step with one active chain passes
    // its operands twice and ignores the second result, so that every step of
    // the kernel runs the same code (fewer copies of it for the instruction cache).
    // The factor rows of a step are read from their slots into rs_d / rs_u, by the step
    // itself or, inside the chains in complex128, already by the previous step before its
    // barrier (the rows do not depend on the chain, so their shared-memory reads leave the
    // critical path of the slower FP64 products: 14 % faster; complex64 steps gained nothing
    // from it and read their rows in the step).
    constexpr bool kPrefetch = sizeof(C) == sizeof(double2);
    C rs_d[NJ], rs_u[NJ];
    bool have_rows = false;
    auto step2 = [&](const C* Sd, const C* td, const C* Su, const C* tu) {
        if (compute) {
            if (!have_rows) {
                load_row<C, NJ>(rs_d, Sd + lofs);
                load_row<C, NJ>(rs_u, Su + lofs);
            }
            dual_rows_r<C, NJ, BT, true, true>(rs_d, rs_u, td + vofs, tu + vofs, nb, vd, vu);
        }
        have_rows = false;
    };
    // the next step's rows, read before this step's barrier
    auto prefetch = [&](const C* S1, const C* S2) {
        if (compute) {
            load_row<C, NJ>(rs_d, S1 + lofs);
            load_row<C, NJ>(rs_u, S2 + lofs);
        }
        have_rows = true;
    };
    // the blocks of a step with chains a (first in load order) and b, either may be off
    auto consume_ab = [&](bool a, bool b, const C*& Sa, const C*& Sb) {
        Sa = Sb = nullptr;
        if (!a && !b) return;
        const C *S1, *S2;
        consume2(a && b, S1, S2);
        Sa = a ? S1 : nullptr;
        Sb = b ? (a ? S2 : S1) : nullptr;
    };
    const bool own1 = rowok && g == 0;                 // BT = 1: the lane that stores a row
    auto owns = [&](int b) -> bool { return BT == 1 ? own1 : (b < nb && rowok && (b & 3) == g); };
    C* const zl = zb + row;                            // this lane's entry of z-buffer row r0, b = 0
    const int zs = BT * W;                             // z-buffer stride between grid rows
    // One chain step of both halves, one code path for the forward, back and separator
    // steps.  S1 is the first active half's block, S2 the second's (S1 again when only
    // one half is active).  Per half h (this lane's row, RHS b), with v the product:
    //   out = az * z[h] + sv * v,   z[h] <- out,   and, if wv[h],
    //   vout[h] = ez * zn[h] + fc * ck[h] * out
    // forward (az 0, sv 1, ez 1, fc -1): z = v, next input b_next - C z;
    // back (az 1, sv -1, ez 0, fc 1): y = z - v, C y to the next row;
    // separator (as back with ck = 1): x = z - v, x to the next separator.
    // The owner lanes read z and zn before the product, off the critical path.
    //   the last step of a half also leaves ps * vout (plus pbase for the up half)
    //   in pv_d / pv_u when pd / pu is set
    //   pf (before the barrier) fetches the next step's rows when the chain has one
    auto gstep = [&](auto&& pf, bool D, bool U, const C* S1, const C* S2, C* zd, C* zu, const C* znd, const C* znu,
                     C ckd, C cku, bool wvd, bool wvu, R az, R sv, R ez, R fc, bool pd = false, bool pu = false,
                     const C* pbase = nullptr, R ps = (R)1) -> bool {
        C pzd[BT], pzu[BT], pnd[BT], pnu[BT];
#pragma unroll
        for (int b = 0; b < BT; ++b) {
            const bool ob = owns(b);
            pzd[b] = (ob && D && az != (R)0) ? zd[b * W] : CT<C>::zero();
            pzu[b] = (ob && U && az != (R)0) ? zu[b * W] : CT<C>::zero();
            pnd[b] = (ob && D && wvd && ez != (R)0) ? znd[b * W] : CT<C>::zero();
            pnu[b] = (ob && U && wvu && ez != (R)0) ? znu[b * W] : CT<C>::zero();
        }
        step2(S1, D ? vin_d : vin_u, S2, U ? vin_u : vin_d);
#pragma unroll
        for (int b = 0; b < BT; ++b)
            if (owns(b)) {
                if (D) {
                    const C out = cadd(cscale(pzd[b], az), cscale(vd[b], sv));
                    zd[b * W] = out;
                    const C vo = cadd(cscale(pnd[b], ez), cscale(cmul(ckd, out), fc));
                    if (wvd) vout_d[b * 64 + row] = vo;
                    if (pd) pv_d[b * 64 + row] = cscale(vo, ps);
                }
                if (U) {
                    const C out = cadd(cscale(pzu[b], az), cscale(vu[b], sv));
                    zu[b * W] = out;
                    const C vo = cadd(cscale(pnu[b], ez), cscale(cmul(cku, out), fc));
                    if (wvu) vout_u[b * 64 + row] = vo;
                    if (pu) pv_u[b * 64 + row] = cadd(pbase ? pbase[b * 64 + row] : CT<C>::zero(), cscale(vo, ps));
                }
            }
        pf();
        return finish();
    };
    C* parts = reinterpret_cast<C*>(A.parts);
    auto pidx = [&](int b, int q, int k) -> int64_t { return (((int64_t)(b0 + b) * Q + q) * kParts + k) * A.Wmax; };
    C* acc2 = reinterpret_cast<C*>(A.acc2);
    auto a2idx = [&](int b, int r) -> int64_t { return ((int64_t)(b0 + b) * imax(NG - 1, 1) + r) * A.Wmax; };
    int* cnt = A.counters + (int64_t)tile * (NG + 1);   // group arrivals [0, NG), level-2 arrivals [NG]
    if (!l2cta) {   // ---- the chunk (the level-2 CTA skips to the level-2 solve)
    // ---- forward elimination: both halves while both have rows, then the longer one
    //   down: z_kd, kd = r0+s; next input b_{kd+1} - C_{kd+1} z_kd (if kd+1 < t)
    //   up:   z_ku, ku = r1-1-s; next input b_{ku-1} - C_ku z_ku (if ku-1 > t)
    for (int s = 0; s < nmx; ++s) {
        const bool D = s < nd, U = s < nu;
        const int ui = m - 1 - s;                          // ku - r0
        const C *S1 = nullptr, *S2 = nullptr;
        if (s == 0 || !kPrefetch) consume2(D && U, S1, S2);   // in order: the down block, then the up block
        auto pf = [&]() {
            if (kPrefetch && s + 1 < nmx) {
                const C *N1, *N2;
                consume2(s + 1 < nd && s + 1 < nu, N1, N2);
                prefetch(N1, N2);
            }
        };
        if (!gstep(pf, D, U, S1, S2, zl + s * zs, zl + ui * zs, zl + (s + 1) * zs, zl + (ui - 1) * zs,
                   cmul(csx_r, ccy[s + 1]), cmul(csx_r, ccy[ui]), r0 + s + 1 < t, r1 - 2 - s > t, (R)0, (R)1,
                   (R)1, (R)-1))
            return;
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
        step2(St, vin_d, St, vin_d);
        const C cd = cpl(t), cu = cpl(t + 1);
#pragma unroll
        for (int b = 0; b < BT; ++b)
            if (owns(b)) {
                zr(t)[b * W + row] = vd[b];
                vout_d[b * 64 + row] = cmul(cd, vd[b]);   // C_t y_t for row t-1
                vout_u[b * 64 + row] = cmul(cu, vd[b]);   // C_{t+1} y_t for row t+1
                if (nd == 0) pv_d[b * 64 + row] = cneg(cmul(cd, vd[b]));              // t = r0
                if (nu == 0) pv_u[b * 64 + row] = csub(rsep[b * 64 + row], cmul(cu, vd[b]));   // t = r1-1
            }
        if (!finish()) return;
    }
    // ---- outward back substitution: y_k = z_k - Sinv_k C y_inner
    //   down: kd = t-1-s, C_kd y_kd to row kd-1;  up: ku = t+1+s, C_{ku+1} y_ku to row ku+1
    // the blocks of back step s (resident: the slots where the forward pass left them)
    auto back_blocks = [&](int s, const C*& S1, const C*& S2) {
        const bool D = s < nd, U = s < nu;
        const int di = nd - 1 - s, ui = nd + 1 + s;
        if (resident) {
            // forward position: down row r0+i at i + min(i, nu); up row r1-1-i at min(i+1, nd) + i
            const C* Sd = D ? reinterpret_cast<const C*>(slots + (size_t)(di + imin(di, nu)) * sb) : nullptr;
            const int i = m - 1 - ui;
            const C* Su = U ? reinterpret_cast<const C*>(slots + (size_t)(imin(i + 1, nd) + i) * sb) : nullptr;
            S1 = D ? Sd : Su;
            S2 = (D && U) ? Su : S1;
        } else {
            consume2(D && U, S1, S2);
        }
    };
    for (int s = 0; s < nmx; ++s) {
        const bool D = s < nd, U = s < nu;
        const int di = nd - 1 - s;              // kd - r0
        const int ui = nd + 1 + s;              // ku - r0
        const C *S1 = nullptr, *S2 = nullptr;
        if (s == 0 || !kPrefetch) back_blocks(s, S1, S2);
        auto pf = [&]() {
            if (kPrefetch && s + 1 < nmx) {
                const C *N1, *N2;
                back_blocks(s + 1, N1, N2);
                prefetch(N1, N2);
            }
        };
        // the last steps leave the parts inputs: -C_r0 y(first) and S r(r1) - C_r1 y(last)
        if (!gstep(pf, D, U, S1, S2, zl + di * zs, zl + ui * zs, nullptr, nullptr, cmul(csx_r, ccy[D ? di : 0]),
                   cmul(csx_r, ccy[U ? ui + 1 : 0]), true, true, (R)1, (R)-1, (R)0, (R)1, s == nd - 1, s == nu - 1,
                   rsep, (R)-1))
            return;
    }
    hold = false;   // the chunk's slots are free from here on: the next refill streams the separator chains
    // ---- chunk solution to global memory
    for (int o = tid; o < m * nb * W; o += blockDim.x) {
        const int c = o % W, b = (o / W) % nb, r = o / (W * nb);
        yrow<C>(A, b0 + b, r0 + r)[c] = zb[(r * BT + b) * W + c];
    }
    if (Q == 0) return;   // every load of the sequence has been consumed
    // ---- separator right-hand-side parts, both in one step:
    //   down chain: A_p     = Rinv_p     (b_s - C_s y(last)),   s = r1      (separator below)
    //   up chain:   B_{p-1} = -Rinv_{p-1} C_{s'+1} y(first),     s' = r0 - 1 (separator above)
    {   // inputs left by the last back steps (or the twist): pv_u = S r(r1) - C_r1 y(last), pv_d = -C_r0 y(first)
        const C *SA, *SB;
        consume_ab(has_below, has_above, SA, SB);
        step2(has_below ? SA : SB, has_below ? pv_u : pv_d, has_above ? SB : SA, has_above ? pv_d : pv_u);
#pragma unroll
        for (int b = 0; b < BT; ++b)
            if (b < nb && rowok && (b & 3) == g) {
                // a level-2 separator's parts go straight into its accumulator (the level-2
                // CTA then reads one value per entry)
                if (has_below) {
                    if (NG > 1 && grp_of(p) < 0) catomic_add(acc2 + a2idx(b, -grp_of(p) - 1) + row, vd[b]);
                    else parts[pidx(b, p, 0) + row] = vd[b];
                }
                if (has_above) {
                    if (NG > 1 && grp_of(p - 1) < 0) catomic_add(acc2 + a2idx(b, -grp_of(p - 1) - 1) + row, vu[b]);
                    else parts[pidx(b, p - 1, 1) + row] = vu[b];
                }
                // the parts as the next step's inputs (vout becomes vin at the barrier)
                vout_d[b * 64 + row] = has_below ? vd[b] : CT<C>::zero();
                vout_u[b * 64 + row] = has_above ? vu[b] : CT<C>::zero();
            }
        if (!finish()) return;
    }
    if (NG > 1) {
        // ---- the chunk's contributions to the level-2 right-hand sides below (dn) and above
        // (up) its group: Q2L/Q2U of separator p times A_p, of separator p-1 times B_{p-1}
        C dn[BT], up[BT];
        auto contrib = [&](bool a, bool b, C (&out)[BT]) {
#pragma unroll
            for (int bb = 0; bb < BT; ++bb) out[bb] = CT<C>::zero();
            if (!a && !b) return;
            const C *SA, *SB;
            consume_ab(a, b, SA, SB);
            // an absent term multiplies the zero vector with the other term's block
            step2(a ? SA : SB, a ? vin_d : vzero, b ? SB : SA, b ? vin_u : vzero);
#pragma unroll
            for (int bb = 0; bb < BT; ++bb) out[bb] = cadd(vd[bb], vu[bb]);
        };
        contrib(q2dnA, q2dnB, dn);
        contrib(q2upA, q2upB, up);
#pragma unroll
        for (int b = 0; b < BT; ++b)
            if (b < nb && rowok && (b & 3) == g) {
                // to the level-2 separator below the group (its index is the group's) and above it;
                // the sums come out in arrival order, so the level-2 right-hand sides agree
                // between runs to rounding, not bitwise
                const int gg = q2dnA || q2upA ? grp_of(p) : grp_of(p - 1);
                if (q2dnA || q2dnB) catomic_add(acc2 + a2idx(b, gg) + row, dn[b]);
                if (q2upA || q2upB) catomic_add(acc2 + a2idx(b, gg - 1) + row, up[b]);
            }
        if (!finish()) return;
        // release: this CTA's parts and contributions (ordered before by the barrier)
        if (tid == 0) asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(cnt + NG) : "memory");
    }
    }   // ---- end of the chunk
    // ---- arrival: the last chunk CTA of group gi (chunks gq0..gq1) solves its separators
    auto arrive = [&](int* ctr, int expect) -> bool {   // after a barrier; true on the last arrival
        if (tid == 0) {
            // release: this CTA's writes (ordered before by the barrier); acquire: the
            // writes every earlier arrival released
            int old;
            asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], 1;" : "=r"(old) : "l"(ctr) : "memory");
            const bool last = old == expect;
            if (last) *ctr = 0;   // next used by a later launch
            flags[0] = last ? 1 : 0;
        }
        __syncthreads();
        if (flags[0]) return true;
        land(consumed);   // not the last: let the copies already issued land before leaving
        return false;
    };
    auto zq = [&](int i) -> C* { return zb + i * BT * W; };
    // one separator step: out_i = z_i - product, stored to z_i and to the chain's next input
    //   first: the step's blocks are consumed here (later steps of a loop have their rows
    //   prefetched by the step before); next: the next step of the loop has blocks for
    //   both halves (2), one (1) or there is none (0)
    auto sep = [&](bool first, int next, bool D, bool U, int qd, int qu, bool pd = false, bool pu = false) -> bool {
        const C *S1 = nullptr, *S2 = nullptr;
        if (first || !kPrefetch) consume2(D && U, S1, S2);
        auto pf = [&]() {
            if (kPrefetch && next > 0) {
                const C *N1, *N2;
                consume2(next == 2, N1, N2);
                prefetch(N1, N2);
            }
        };
        const C one = CT<C>::from(make_double2(1.0, 0.0));
        return gstep(pf, D, U, S1, S2, zq(qd) + row, zq(qu) + row, nullptr, nullptr, one, one, true, true, (R)1,
                     (R)-1, (R)0, (R)1, pd, pu);
    };
    auto nxt = [](int s, int a, int b) -> int { return (s + 1 < a ? 1 : 0) + (s + 1 < b ? 1 : 0); };
    // Twisted solve of n separators in the load order of chain_order; a_i is in
    // zq(i), a_0 / a_{n-1} in vin_d / vin_u.
    auto chain = [&](int n) -> bool {
        const int tq = (n - 1) / 2;
        const int fd = imax(tq - 1, 0), fu = imax(n - 2 - tq, 0);   // forward steps
        const int bd = tq, bu = n - 1 - tq;                          // back steps
        // forward: z_i = a_i - E_i z_outer, down i = 1..tq-1, up i = n-2..tq+1
        for (int s = 0; s < imax(fd, fu); ++s)
            if (!sep(s == 0, nxt(s, fd, fu), s < fd, s < fu, 1 + s, n - 2 - s)) return false;
        // twist: x_tq = a_tq - E_tq z_{tq-1} - F_tq z_{tq+1}
        for (int o = tid; o < nb * W; o += blockDim.x) {
            const int c = o % W, b = o / W;
            if (tq >= 1) vin_d[b * 64 + c] = zq(tq - 1)[b * W + c];
            if (tq <= n - 2) vin_u[b * 64 + c] = zq(tq + 1)[b * W + c];
        }
        __syncthreads();
        {
            const bool he = tq >= 1, hf = tq <= n - 2;
            const C *Se, *Sf;
            consume_ab(he, hf, Se, Sf);
            step2(he ? Se : Sf, he ? vin_d : vin_u, hf ? Sf : Se, hf ? vin_u : vin_d);
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
                    if (tq == 0) pv_d[b * 64 + row] = x;        // x_0
                    if (tq == n - 1) pv_u[b * 64 + row] = x;    // x_{n-1}
                }
            if (!finish()) return false;
        }
        // back: x_i = z_i - F_i x_inner, down i = tq-1..0, up i = tq+1..n-1; the last
        // steps leave x_0 in pv_d and x_{n-1} in pv_u
        for (int s = 0; s < imax(bd, bu); ++s)
            if (!sep(s == 0, nxt(s, bd, bu), s < bd, s < bu, tq - 1 - s, tq + 1 + s, s == bd - 1, s == bu - 1))
                return false;
        return true;
    };
    // right-hand sides a_i = sum of the parts of separator slot(i), two entries
    // per thread with their loads in flight together
    auto load_a = [&](int n, int lvl) {   // compute warps only: the producer warp streams blocks meanwhile
        if (!compute) return;
        const int tot = n * nb * W;
        for (int o0 = tid; o0 < tot; o0 += 4 * ptid) {
            C v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int o = o0 + u * ptid;
                if (o < tot) {
                    const int c = o % W, b = (o / W) % nb, i = o / (W * nb);
                    if (lvl == 1) {
                        const int64_t pb = pidx(b, q0 + i, 0) + c;
                        v[u] = cadd(__ldcg(parts + pb), __ldcg(parts + pb + A.Wmax));
                    } else {   // the whole right-hand side, summed by the chunks; zero for the next launch
                        C* ap = acc2 + a2idx(b, i) + c;
                        v[u] = __ldcg(ap);
                        *ap = CT<C>::zero();
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int o = o0 + u * ptid;
                if (o < tot) {
                    const int c = o % W, b = (o / W) % nb, i = o / (W * nb);
                    zb[(i * BT + b) * W + c] = v[u];
                    if (i == 0) vin_d[b * 64 + c] = v[u];
                    if (i == n - 1) vin_u[b * 64 + c] = v[u];
                }
            }
        }
        asm volatile("bar.sync 1, %0;" ::"r"(ptid) : "memory");
    };
    // ---- level 1: the group's separators q0 .. q1-1 with the level-2 separators at zero,
    //      by the last chunk of the group to arrive
    if (!l2cta) {
        if (!arrive(&cnt[gi], n1)) return;
        if (pwarp) {   // the rest of the group chain streams in
            cap = nload;
            refill();
        }
        load_a(n1, 1);
        if (!chain(n1)) return;
        for (int o = tid; o < n1 * nb * W; o += blockDim.x) {
            const int c = o % W, b = (o / W) % nb, i = o / (W * nb);
            yrow<C>(A, b0 + b, A.g.r1[q0 + i])[c] = zb[(i * BT + b) * W + c];
        }
        return;
    }
    // ---- level 2 (the level-2 CTA): once every chunk has added its contributions
    if (tid == 0) {
        const unsigned* c2 = reinterpret_cast<const unsigned*>(cnt + NG);
        const unsigned target = (unsigned)P;   // every chunk's contributions are in
        unsigned v = 0;
        uint32_t it = 0;
        for (; it < kWaitLimit; ++it) {
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(c2) : "memory");
            if (v >= target) break;
            __nanosleep(64);
        }
        const bool ok = v >= target;
        if (ok) cnt[NG] = 0;   // next used by a later launch (every chunk of this one has arrived)
        flags[0] = ok ? 0 : 1;
    }
    __syncthreads();
    if (flags[0]) {
        abort_wait();
        return;
    }
    load_a(n2, 2);
    if (!chain(n2)) return;
    for (int o = tid; o < n2 * nb * W; o += blockDim.x) {
        const int c = o % W, b = (o / W) % nb, i = o / (W * nb);
        yrow<C>(A, b0 + b, A.g.r1[i < 64 ? l2s[i] : A.g.gq1[i]])[c] = zb[(i * BT + b) * W + c];
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

// Output columns of many finished strip solves in one launch (grid: chunks x
// strips x RHS tiles; throughput, not latency).  The final values of the chunk's
// two separators first: the chain kernel's values, for grouped separators
// corrected by the level-2 spikes, x_q = y2_q - GT2_q x2_{gi-1} - GB2_q x2_{gi}.
// Then row k of chunk p gets x_k = y_k - GT_p(k) x_{p-1} - GB_p(k) x_p, the
// separator row below the chunk its final value; x (plus the base field) goes to
// the strip's output columns.  8 lanes per value; the row tasks two per group at a
// time with all their loads in flight together.
template <typename C>
__global__ void __launch_bounds__(256, 2) k_sweep_output(OutArgs O, const C* __restrict__ GT,
                                                         const C* __restrict__ GB, const C* __restrict__ GT2,
                                                         const C* __restrict__ GB2) {
    __shared__ C xsv[2][4][64];   // separator above / below, per RHS (Bt <= 4)
    const int ntile = (O.B + O.Bt - 1) / O.Bt;
    const int nitem = O.g.P * O.nstrip * ntile;
    for (int item = blockIdx.x; item < nitem; item += gridDim.x) {   // (chunk, strip, RHS tile)
        __syncthreads();   // xsv of the previous item consumed
        const int p = item % O.g.P;
        const int j = O.jlo + (item / O.g.P) % O.nstrip;
        const int b0 = (item / (O.g.P * O.nstrip)) * O.Bt;
        const int nb = imin(O.Bt, O.B - b0);
        const StripDev st = O.g.strips[j];
        const int W = st.W, SL = spld(W);
        const int P = O.g.P, NG = O.g.G;
        const int off = st.lo - st.lpml;
        const int olo = imax(st.olo[O.dir] - off, 0), ohi = imin(st.ohi[O.dir] - off, W - 1);
        const int nout = ohi - olo + 1;
        if (nout <= 0) continue;
        const int4 m0 = O.g.cmeta[2 * p], m1 = O.g.cmeta[2 * p + 1];
        const int r0 = m0.x, r1 = m0.y, m = r1 - r0;
        const C* Y = reinterpret_cast<const C*>(O.ybuf) + (int64_t)j * O.ystride;
        const bool above = p > 0, below = p < P - 1;
        const int tid = threadIdx.x, w = tid >> 5, l = tid & 31, g = tid & 7, grp = tid >> 3, ngrp = blockDim.x >> 3;
        auto yr = [&](int b, int k) { return Y + ((int64_t)(b0 + b) * O.g.Ny + k) * O.Wmax; };
        // ---- final separator values
        const int srow[2] = {r0 - 1, r1}, sg[2] = {m0.z, m0.w}, sra[2] = {m1.x, m1.z}, srb[2] = {m1.y, m1.w};
        for (int side = 0; side < 2; ++side) {
            const bool on = side == 0 ? above : below;
            const int gi = on ? sg[side] : -1;
            for (int b = 0; b < nb; ++b) {
                const C* y = yr(b, on ? srow[side] : r0);
                if (gi < 0) {   // no separator, a level-2 separator or a single group: already final
                    for (int c = tid; c < 64; c += blockDim.x) xsv[side][b][c] = (on && c < W) ? y[c] : CT<C>::zero();
                    continue;
                }
                const bool up = gi > 0, dn = gi < NG - 1;
                const int64_t o2 = st.red + (int64_t)(side == 0 ? p - 1 : p) * st.bs;
                C xa[8], xb[8];
                lane_vec(xa, yr(b, up ? sra[side] : r0), up, g, W);
                lane_vec(xb, yr(b, dn ? srb[side] : r0), dn, g, W);
                for (int base = w * 4; base < 64; base += (blockDim.x >> 5) * 4) {   // warp-uniform trip count
                    const int c = base + (l >> 3);
                    const int cc = imin(c, W - 1);
                    const C sum = spike_dot2(GT2 + o2 + (int64_t)cc * SL, xa, up, GB2 + o2 + (int64_t)cc * SL, xb, dn, g, W);
                    if (g == 0) xsv[side][b][c] = c < W ? csub(y[c], sum) : CT<C>::zero();
                }
            }
        }
        __syncthreads();
        auto at = [&](int b, int k, int c) { return ((int64_t)(b0 + b) * O.g.Ny + k) * O.g.Nx + off + c; };
        if (below)   // the separator row below the chunk: its final value
            for (int o = tid; o < nb * nout; o += blockDim.x) {
                const int b = o / nout, c = olo + o % nout;
                double2 v = to_d2(xsv[1][b][c]);
                if (O.base) v = cadd(v, O.base[at(b, r1, c)]);
                O.dst[at(b, r1, c)] = v;
            }
        const int ntask = m * nout;
        for (int b = 0; b < nb; ++b) {
            C xa[8], xb[8];
            lane_vec(xa, xsv[0][b], above, g, W);
            lane_vec(xb, xsv[1][b], below, g, W);
            for (int t0 = 0; t0 < ntask; t0 += 2 * ngrp) {   // uniform trip count: every lane shuffles
                int kk[2], c[2];
                bool live[2];
                C sa[2][8], sb[2][8], y[2];
                double2 bv[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {   // loads of both tasks first
                    const int t = t0 + u * ngrp + grp;
                    live[u] = t < ntask;
                    const int tc = imin(t, ntask - 1);
                    kk[u] = tc / nout;
                    c[u] = olo + tc % nout;
                    const int k = r0 + kk[u];
                    const int64_t ro = st.fac + (int64_t)k * st.bs + (int64_t)c[u] * SL;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int a = g + 8 * i;
                        sa[u][i] = (above && a < W) ? GT[ro + a] : CT<C>::zero();
                        sb[u][i] = (below && a < W) ? GB[ro + a] : CT<C>::zero();
                    }
                    y[u] = yr(b, k)[c[u]];
                    bv[u] = O.base ? O.base[at(b, k, c[u])] : make_double2(0.0, 0.0);
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    C s0 = CT<C>::zero(), s1 = CT<C>::zero();
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        s0 = cfma(sa[u][i], xa[i], s0);
                        s1 = cfma(sb[u][i], xb[i], s1);
                    }
                    C sum = cadd(s0, s1);
#pragma unroll
                    for (int o = 1; o <= 4; o <<= 1) {
                        sum.x += __shfl_xor_sync(0xffffffffu, sum.x, o);
                        sum.y += __shfl_xor_sync(0xffffffffu, sum.y, o);
                    }
                    if (live[u] && g == 0) O.dst[at(b, r0 + kk[u], c[u])] = cadd(to_d2(csub(y[u], sum)), bv[u]);
                }
            }
        }
    }
}

// ------------------------------------------------------------------ host
// Bytes of the separator-parts region of a strip solve ([B][P-1][kParts][Wmax]); the
// level-2 accumulators ([B][G-1][Wmax], sized for G - 1 <= P) follow it.
size_t sweep_parts_bytes(int P, int B, int Wmax, size_t esize) {
    return (size_t)B * std::max(P - 1, 1) * kParts * Wmax * esize;
}
size_t sweep_parts_total_bytes(int P, int B, int Wmax, size_t esize) {
    return sweep_parts_bytes(P, B, Wmax, esize) + sweep_parts2_bytes(P, B, Wmax, esize);
}
size_t sweep_parts2_bytes(int P, int B, int Wmax, size_t esize) { return (size_t)B * std::max(P, 1) * Wmax * esize; }

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
    A.Q2L = g.G > 1 ? pool[11] : nullptr;
    A.Q2U = g.G > 1 ? pool[12] : nullptr;
    A.ybuf = wk.ybuf;
    A.parts = wk.parts;
    A.acc2 = reinterpret_cast<char*>(wk.parts) + sweep_parts_bytes(g.P, wk.B, wk.Wmax, sizeof(C));
    A.has_prev = 0;
    A.pybuf = wk.pybuf;
    A.GT = pool[1];
    A.GB = pool[2];
    A.GT2 = pool[6];
    A.GB2 = pool[7];
    A.XF = pool[10];
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

bool strip_solve_fits(const StripDev& st, int zrows, size_t esize) {
    int Bt, ring;
    size_t smem;
    return esize == sizeof(float2) ? plan<float2>(st, zrows, 1, Bt, ring, smem)
                                   : plan<double2>(st, zrows, 1, Bt, ring, smem);
}

// Shared-memory limit of every strip-solve instantiation (this also loads the module).
template <typename C>
static cudaError_t chunk_kernel_attrs() {
    for (auto fn : {k_sweep_chunk<C, 8, 1>, k_sweep_chunk<C, 10, 1>, k_sweep_chunk<C, 12, 1>,
                    k_sweep_chunk<C, 14, 1>, k_sweep_chunk<C, 16, 1>, k_sweep_chunk<C, 8, 4>,
                    k_sweep_chunk<C, 10, 4>, k_sweep_chunk<C, 12, 4>, k_sweep_chunk<C, 14, 4>,
                    k_sweep_chunk<C, 16, 4>}) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t preload_sweep_kernels() {
    cudaError_t e = chunk_kernel_attrs<float2>();
    if (e == cudaSuccess) e = chunk_kernel_attrs<double2>();
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_sweep_output<float2>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_sweep_output<double2>);
    return e;
}

template <typename C>
cudaError_t launch_strip_solve(const Geom& g, int j, const StripDev& st, const StripDev* pst,
                               const SweepStep& step, const SweepWork& wk, void* const* pool, cudaStream_t s,
                               KernelTimer* tm) {
    int Bt, ring;
    size_t smem;
    if (!plan<C>(st, wk.zrows, wk.B, Bt, ring, smem)) return cudaErrorInvalidConfiguration;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = chunk_kernel_attrs<C>();
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    SweepArgs A = make_args<C>(g, st, step, wk, pool, Bt, ring);
    if (pst && step.prev >= 0) {
        A.has_prev = 1;
        A.pst = *pst;
    }
    const int ntile = (wk.B + Bt - 1) / Bt;
    // consecutive strip solves with programmatic stream serialisation (see pdl_wait)
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = wk.pdl ? 1 : 0;
    auto config = [&](dim3 grid, int nthr, size_t bytes) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = dim3(nthr);
        cfg.dynamicSmemBytes = bytes;
        cfg.stream = s;
        cfg.attrs = pdl;
        cfg.numAttrs = 1;
        return cfg;
    };
    cudaError_t err;
    {
        void (*kfn)(SweepArgs) = nullptr;
#define HELM_CHUNK_FN(NJ) kfn = Bt == 1 ? k_sweep_chunk<C, NJ, 1> : k_sweep_chunk<C, NJ, 4>
        switch (st.nj) {
            case 8: HELM_CHUNK_FN(8); break;
            case 10: HELM_CHUNK_FN(10); break;
            case 12: HELM_CHUNK_FN(12); break;
            case 14: HELM_CHUNK_FN(14); break;
            default: HELM_CHUNK_FN(16); break;
        }
#undef HELM_CHUNK_FN
        // compute warps + the producer warp; with separator groups one more CTA for level 2
        const cudaLaunchConfig_t cfg = config(dim3(g.P + (g.G > 1 ? 1 : 0), ntile), 32 * ((st.W + 7) / 8 + 1), smem);
        TimedLaunch t(tm, "sweep_chunk", s);
        err = cudaLaunchKernelEx(&cfg, kfn, A);
    }
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

template <typename C>
cudaError_t launch_outputs(const OutArgs& O, void* const* pool, cudaStream_t s, KernelTimer* tm) {
    if (O.nstrip <= 0) return cudaSuccess;
    TimedLaunch t(tm, "sweep_output", s);
    const int nitem = O.g.P * O.nstrip * ((O.B + O.Bt - 1) / O.Bt);
    const int grid = O.maxcta > 0 ? imin(nitem, O.maxcta) : nitem;
    k_sweep_output<C><<<grid, 256, 0, s>>>(O, (const C*)pool[1], (const C*)pool[2], (const C*)pool[6],
                                         (const C*)pool[7]);
    return cudaGetLastError();
}

template cudaError_t launch_outputs<float2>(const OutArgs&, void* const*, cudaStream_t, KernelTimer*);
template cudaError_t launch_outputs<double2>(const OutArgs&, void* const*, cudaStream_t, KernelTimer*);

template cudaError_t launch_strip_solve<float2>(const Geom&, int, const StripDev&, const StripDev*,
                                                const SweepStep&, const SweepWork&, void* const*, cudaStream_t,
                                                KernelTimer*);
template cudaError_t launch_strip_solve<double2>(const Geom&, int, const StripDev&, const StripDev*,
                                                 const SweepStep&, const SweepWork&, void* const*, cudaStream_t,
                                                 KernelTimer*);

}  // namespace helm
