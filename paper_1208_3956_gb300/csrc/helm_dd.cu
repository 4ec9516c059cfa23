// Host side of the helm_dd C ABI: problem set-up, PML tables, strip geometry,
// device memory, the double-sweep driver, flexible GMRES and the misfit
// gradient.  All arithmetic on fields runs in the kernels of factor.cu,
// sweep.cu and field.cu; the host computes O(N) one-dimensional tables and the
// O(restart^2) Hessenberg/Givens work of GMRES.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <complex>
#include <functional>
#include <string>
#include <vector>

#include "helm_dd.h"
#include "internal.h"

using namespace helm;
typedef std::complex<double> cd;

namespace {

// ---- PML (Section 2.1): d/dx -> (1 + i sigma/omega)^-1 d/dx, quadratic profile.
struct Pml {
    double sigma0 = 0.0;
    int w = 0;
    double h = 1.0, omega = 1.0;
    // alpha at a point whose distance into the layer is d2 half-steps (d = d2 h / 2)
    cd alpha(int d2) const {
        if (w <= 0 || d2 <= 0) return cd(1.0, 0.0);
        const double L = w * h;
        const double d = std::min(0.5 * d2 * h, L);
        const double s = sigma0 * (d / L) * (d / L);
        return 1.0 / cd(1.0, s / omega);
    }
};

double pml_sigma0(double c_ref, int w, double h) {
    if (w <= 0) return 0.0;
    return 3.0 * c_ref * log(1.0e6) / (2.0 * w * h);
}

// alpha on a padded axis of Np points with a w-point layer at both ends, as a
// function of position in half-steps x2 (integer point i at x2 = 2i, half point
// i+1/2 at x2 = 2i+1).  Interfaces at x_{w-1/2} and x_{Np-w-1/2}.
cd axis_alpha_at(const Pml& p, int Np, int x2) {
    if (p.w <= 0) return cd(1.0, 0.0);
    const int lo2 = 2 * p.w - 1, hi2 = 2 * (Np - p.w) - 1;
    const int d2 = std::max(std::max(lo2 - x2, x2 - hi2), 0);
    return p.alpha(d2);
}

}  // namespace

struct helm_dd {
    // problem
    int dim = 2;
    int64_t n[3] = {1, 1, 1};
    int64_t N[3] = {1, 1, 1};
    double h = 1.0, omega = 1.0, c_ref = 0.0;
    int w_outer = 0, w_sub = 0, J = 1, P_req = 0, G_req = 0;
    int panel = 0;   // most right-hand sides per internal panel of solve / gradient (0: as many as fit)
    int transmission = HELM_TRANSMISSION_PML;
    int sweep = HELM_SWEEP_DOUBLE;
    int nsm = 0;                        // SMs of the device (chunk count of concurrent sweeps)
    // concurrent sweeps: the downward sequence and the total-field corrections run on two
    // more streams, ordered by events
    cudaStream_t cstream[2] = {nullptr, nullptr};
    cudaEvent_t cev[4] = {nullptr, nullptr, nullptr, nullptr};
    double2* d_rab = nullptr;   // Robin a/b per interface and row ([J][Ny]), Robin transmission only
    helm_prec prec = HELM_PREC_FP64;
    std::vector<double> c;
    // geometry
    std::vector<int> beta;
    std::vector<StripDev> strips;
    int P = 1, G = 1, Wmax = 0;
    std::vector<int> r0, r1, rowmap;
    std::vector<int> gq0, gq1, sepmap;   // separator groups (second level of nested dissection)
    std::vector<cd> gx_int, gx_half, gy_int, gy_half, gz_int, gz_half;
    // device
    cudaStream_t stream = nullptr, own_stream = nullptr;
    // the output passes run beside the strip solves: a low-priority stream and its events
    cudaStream_t side = nullptr;
    cudaEvent_t ev_main = nullptr, ev_side = nullptr;
    Geom geom{};
    double* d_c = nullptr;
    double* d_k2 = nullptr;
    double2* d_tab = nullptr;       // global axis tables + per-strip x tables
    void* d_ct = nullptr;           // working-precision sweep tables
    int* d_counters = nullptr;      // per-tile arrival counters of the sweep ([kMaxTiles][G+1])
    size_t counter_bytes = 0;
    int zrows = 1;
    StripDev* d_strips = nullptr;
    int* d_ints = nullptr;          // cmeta (8 per chunk) | r0 | r1 | rowmap | gq0 | gq1 | sepmap
    // factors: Sinv GT GB (per grid row), Rinv E F GT2 GB2 P2L P2U (per separator), transfer composites,
    // level-2 contributions Q2L Q2U (per separator)
    void* d_pool[13] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                        nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int* d_status = nullptr;
    // 3-D strips: s_x s_z per block entry (working precision) and its per-strip offsets,
    // the offset of s_z in d_ct, the y-couplings -alpha_y(y_{k-1/2})/h^2 and the row
    // stride of the strip right-hand-side / solution buffers
    void* d_slab_sxz = nullptr;
    std::vector<int64_t> slab_sxz_off;
    int64_t ct_sz = 0;
    std::vector<double2> slab_cy;
    int slab_ld = 0;
    size_t esize = 16;
    bool factored = false;
    bool prepared = false;
    bool dev_ready = false;
    void* noalloc_base = nullptr;   // device address of the no-allocation scratch array
    // workspaces
    struct Ws { void* p = nullptr; size_t bytes = 0; };
    Ws ws_V, ws_G, ws_Y, ws_parts, ws_io_in, ws_io_out, ws_io_aux, ws_kry, ws_small, ws_grad, ws_red;
    // interface lines of the reduced space (Section 2.3): padded columns beta_j+1, beta_j+2
    std::vector<int> icols;
    int* d_icols = nullptr;
    KernelTimer timer;
    std::string err;
};

namespace {

constexpr int kMaxTiles = 4096;   // RHS tiles of one sweep launch (4 RHS per tile)

helm_status fail(helm_dd* h, helm_status s, const std::string& msg) {
    if (h) h->err = msg;
    return s;
}
helm_status fail_cuda(helm_dd* h, const char* what, cudaError_t e) {
    return fail(h, e == cudaErrorMemoryAllocation ? HELM_ENOMEM : HELM_ECUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}
#define CK(h, call)                                                    \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return fail_cuda((h), #call, e_);       \
    } while (0)

helm_status ws_reserve(helm_dd* h, helm_dd::Ws& w, size_t bytes) {
    if (w.bytes >= bytes) return HELM_OK;
    if (w.p) cudaFree(w.p);
    w.p = nullptr;
    w.bytes = 0;
    cudaError_t e = cudaMalloc(&w.p, bytes);
    if (e != cudaSuccess) { cudaGetLastError(); return fail_cuda(h, "cudaMalloc(workspace)", e); }
    w.bytes = bytes;
    return HELM_OK;
}
void ws_free(helm_dd::Ws& w) {
    if (w.p) cudaFree(w.p);
    w.p = nullptr;
    w.bytes = 0;
}

// complex128 device fields are read with 16-byte accesses
bool misaligned16(const void* p) { return ((uintptr_t)p & 15) != 0; }

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int64_t nvol(const helm_dd* h) { return h->N[0] * h->N[1] * h->N[2]; }

// Strip geometry (Section 2.1, Eq. grid_A_j) and its x tables.
void build_geometry(helm_dd* h) {
    const int Nx = (int)h->N[0];
    const int nx = (int)h->n[0];
    h->beta.assign(h->J + 1, 0);
    for (int j = 0; j <= h->J; ++j) h->beta[j] = h->w_outer - 1 + (int)floor((double)j * nx / h->J + 0.5);
    h->beta[0] = -1;
    h->beta[h->J] = Nx - 1;
    h->strips.assign(h->J, StripDev{});
    h->Wmax = 0;
    for (int j = 0; j < h->J; ++j) {
        StripDev& s = h->strips[j];
        s.j = j;
        s.lo = h->beta[j] + 1;
        s.hi = (j < h->J - 1) ? h->beta[j + 1] + 1 : Nx - 1;
        // Robin transmission (Section 4.4): no added layers, the same physical columns
        const bool robin = h->transmission == HELM_TRANSMISSION_ROBIN;
        s.lpml = j > 0 && !robin ? h->w_sub : 0;
        s.rpml = j < h->J - 1 && !robin ? h->w_sub : 0;
        s.W = s.lpml + (s.hi - s.lo + 1) + s.rpml;
        h->Wmax = std::max(h->Wmax, s.W);
    }
    h->icols.clear();
    for (int j = 1; j < h->J; ++j) {
        h->icols.push_back(h->beta[j] + 1);
        h->icols.push_back(h->beta[j] + 2);
    }
}

void build_tables(helm_dd* h) {
    Pml po;
    po.w = h->w_outer;
    po.h = h->h;
    po.omega = h->omega;
    po.sigma0 = pml_sigma0(h->c_ref, h->w_outer, h->h);
    auto axis = [&](int Np, std::vector<cd>& ai, std::vector<cd>& ah) {
        ai.resize(Np);
        ah.resize(Np + 1);
        for (int i = 0; i < Np; ++i) ai[i] = axis_alpha_at(po, Np, 2 * i);
        for (int m = 0; m <= Np; ++m) ah[m] = axis_alpha_at(po, Np, 2 * m - 1);
    };
    axis((int)h->N[0], h->gx_int, h->gx_half);
    axis((int)h->N[1], h->gy_int, h->gy_half);
    if (h->dim == 3) axis((int)h->N[2], h->gz_int, h->gz_half);
    else { h->gz_int.assign(1, cd(1.0, 0.0)); h->gz_half.assign(2, cd(1.0, 0.0)); }
}

// alpha along x at strip-local half-step position x2 (column c at 2c, half point
// m-1/2 at 2m-1): inside an added layer measured from the subdomain interface,
// otherwise the global table.
cd strip_alpha_at(const helm_dd* h, const StripDev& s, int x2) {
    const int g2 = x2 + 2 * (s.lo - s.lpml);          // padded half-step position
    const int lo_if2 = 2 * s.lo - 1, hi_if2 = 2 * s.hi + 1;
    Pml ps;
    ps.w = h->w_sub;
    ps.h = h->h;
    ps.omega = h->omega;
    ps.sigma0 = pml_sigma0(h->c_ref, h->w_sub, h->h);
    if (s.lpml > 0 && g2 < lo_if2) return ps.alpha(lo_if2 - g2);
    if (s.rpml > 0 && g2 > hi_if2) return ps.alpha(g2 - hi_if2);
    Pml po = ps;
    po.w = h->w_outer;
    po.sigma0 = pml_sigma0(h->c_ref, h->w_outer, h->h);
    return axis_alpha_at(po, (int)h->N[0], g2);
}

void chunk_layout(helm_dd* h) {
    const int Ny = (int)h->N[1];
    // built-in: a strip solve takes about Ny/P (chunk) + P/G (separator group) + G
    // (level-2 system) dependent steps; G ~ sqrt(P) and P ~ Ny^(2/3) balance them.  The
    // factor 0.93 (fewer, longer chunks) is the measured optimum on a 1055-row grid,
    // where the chunk steps are slightly cheaper than the separator steps.
    int P = h->P_req > 0 ? h->P_req : std::max(1, (int)lround(0.93 * pow((double)Ny, 2.0 / 3.0)));
    // A panel of B > 4 right-hand sides (set before the factorisation) runs each strip
    // solve as ceil(B/4) tiles of P+1 CTAs (one SM each).  Once the tiles exceed one wave
    // of the SMs they run one after another, so the built-in count drops to the P whose
    // tiles all fit one wave, but not below a sixth of it (longer chunk chains).  On 1055
    // rows this halves the time per right-hand side at B = 32 (P = 18 against 96).
    if (h->P_req == 0 && h->panel > 4 && h->nsm > 0) {
        const int tiles = (h->panel + 3) / 4;
        P = std::min(P, std::max(h->nsm / tiles - 1, (P + 5) / 6));
    }
    // concurrent sweeps run three strip solves side by side (one CTA per chunk and SM, and
    // one for the level-2 system)
    if (h->P_req == 0 && h->sweep == HELM_SWEEP_CONCURRENT && h->nsm >= 6) P = std::min(P, h->nsm / 3 - 1);
    P = std::min(P, (Ny + 1) / 2);
    h->P = std::max(P, 1);
    const int rows = Ny - (h->P - 1);
    const int base = rows / h->P, rem = rows % h->P;
    h->r0.assign(h->P, 0);
    h->r1.assign(h->P, 0);
    h->rowmap.assign(Ny, 0);
    int k = 0;
    for (int p = 0; p < h->P; ++p) {
        h->r0[p] = k;
        h->r1[p] = k + base + (p < rem ? 1 : 0);
        for (int r = h->r0[p]; r < h->r1[p]; ++r) h->rowmap[r] = p;
        k = h->r1[p];
        if (p < h->P - 1) { h->rowmap[k] = -(p + 1); k += 1; }
    }
    // Separator groups: the Q = P-1 separators are cut by G-1 level-2 separators
    // into G groups of consecutive separators.  The solve of the separator system
    // then takes about Q/G + G dependent steps instead of Q; G ~ sqrt(Q) balances
    // the two.  Every group keeps at least one separator.
    const int Q = h->P - 1;
    int G = h->G_req > 0 ? h->G_req : (Q >= 6 ? (int)lround(sqrt((double)Q)) : 1);
    G = std::max(1, std::min(G, (Q + 1) / 2));
    // the level-2 factorisation needs a fourth W x W buffer in shared memory
    if (factor_smem_bytes(h->Wmax, h->esize, 4) > kFactorSmemMax) G = 1;
    h->G = G;
    const int nsep = Q - (G - 1);
    const int gbase = G > 0 ? nsep / G : 0, grem = G > 0 ? nsep % G : 0;
    h->gq0.assign(G, 0);
    h->gq1.assign(G, 0);
    h->sepmap.assign(std::max(Q, 1), 0);
    int q = 0;
    for (int gi = 0; gi < G; ++gi) {
        h->gq0[gi] = q;
        h->gq1[gi] = q + gbase + (gi < grem ? 1 : 0);
        for (int i = h->gq0[gi]; i < h->gq1[gi]; ++i) h->sepmap[i] = gi;
        q = h->gq1[gi];
        if (gi < G - 1) { h->sepmap[q] = -(gi + 1); q += 1; }
    }
}

// Row stride of the strip-solution and parts buffers: even, so that every row
// starts 16-byte aligned for bulk copies.
int work_stride(const helm_dd* h) { return (h->Wmax + 1) & ~1; }

// one set per stream that runs strip solves (three for concurrent sweeps)
int sweep_streams(const helm_dd* h) { return h->sweep == HELM_SWEEP_CONCURRENT ? 3 : 1; }
size_t counter_set_bytes(const helm_dd* h) { return (size_t)kMaxTiles * (h->G + 1) * sizeof(int); }
size_t counter_bytes(const helm_dd* h) { return counter_set_bytes(h) * sweep_streams(h); }

double2 to_d2h(cd v) { return make_double2(v.real(), v.imag()); }

}  // namespace

// ------------------------------------------------------------------------
// Scratch of the preconditioner application that allocates nothing.
//
// Some callers cannot let the library allocate device memory while they run:
// programs that hand all device memory to their own pool allocator and forbid
// any other allocation, programs running so close to the memory limit that a
// late workspace allocation could fail mid-run, and latency-critical loops in
// which cudaMalloc / cudaFree would stall the whole device.  For them the
// work buffers of the double sweep come from one file-scope device array.  The
// CUDA runtime loads it (and takes its memory) on a device when this file's
// module is first used there, which ensure_device forces at a handle's first
// device use; it is held until the process exits.
// ------------------------------------------------------------------------
static constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;   // 64 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
constexpr int kNoAllocMaxDevices = 64;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};   // device address of the array, per device

// Device address of the scratch array on the current device.  The array's name
// is only a host-side stand-in, so the address is looked up once per device
// (with that device current) and cached.  Under lazy module loading the lookup
// is what loads the array onto the device.
cudaError_t noalloc_scratch(void** ptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *ptr = g_noalloc_ptr[dev];
    return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// First device use of a handle: stream, medium upload and k^2 (a1).  Creating
// a handle touches no GPU, so its host-side geometry is usable without one.
helm_status ensure_device(helm_dd* h) {
    if (h->dev_ready) return HELM_OK;
    if (!h->own_stream) CK(h, cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
    if (!h->stream) h->stream = h->own_stream;
    {
        int dev = 0;
        CK(h, cudaGetDevice(&dev));
        CK(h, cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev));
    }
    for (auto& cs : h->cstream)
        if (!cs) CK(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    for (auto& ev : h->cev)
        if (!ev) CK(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    if (!h->side) {
        int lo = 0, hi = 0;
        CK(h, cudaDeviceGetStreamPriorityRange(&lo, &hi));   // lo: the lowest priority
        CK(h, cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, lo));
        CK(h, cudaEventCreateWithFlags(&h->ev_main, cudaEventDisableTiming));
        CK(h, cudaEventCreateWithFlags(&h->ev_side, cudaEventDisableTiming));
    }
    // Everything a later call launches is loaded now, where allocation is expected:
    // the no-allocation scratch array (its address cached per device) and the
    // modules of the sweep, slab and grid kernels.
    CK(h, noalloc_scratch(&h->noalloc_base));
    CK(h, preload_sweep_kernels());
    CK(h, preload_slab_kernels());
    CK(h, preload_field_kernels());
    const int64_t nint = (int64_t)h->c.size();
    CK(h, cudaMalloc(&h->d_c, nint * sizeof(double)));
    CK(h, cudaMalloc(&h->d_k2, nvol(h) * sizeof(double)));
    CK(h, cudaMalloc(&h->d_status, sizeof(int)));
    CK(h, cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream));
    CK(h, cudaMemcpyAsync(h->d_c, h->c.data(), nint * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(h, launch_k2(h->d_c, h->d_k2, h->dim, (int)h->n[0], (int)h->n[1], (int)h->n[2], h->w_outer, h->omega,
                    h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->dev_ready = true;
    return HELM_OK;
}

// Build the PML tables, strip geometry and chunk layout and upload them; fills
// h->geom.  Idempotent until helm_dd_set_chunks / set_pml_speed change inputs.
helm_status prepare_geom(helm_dd* h) {
    helm_status ds = ensure_device(h);
    if (ds != HELM_OK) return ds;
    build_tables(h);
    chunk_layout(h);
    std::vector<cd> tabs;
    auto append = [&](const std::vector<cd>& v) { tabs.insert(tabs.end(), v.begin(), v.end()); };
    append(h->gx_int);
    append(h->gx_half);
    append(h->gy_int);
    append(h->gy_half);
    append(h->gz_int);
    append(h->gz_half);
    // stencil entries per axis: {-a(i) a(i-1/2), a(i) (a(i-1/2) + a(i+1/2)), -a(i) a(i+1/2)} / h^2,
    // and the index range where they are exactly {-1, 2, -1} / h^2
    const double ih2s = 1.0 / (h->h * h->h);
    int frange[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    int64_t stc_off[3] = {0, 0, 0};
    auto stencil_axis = [&](int a, const std::vector<cd>& ai, const std::vector<cd>& ah) {
        stc_off[a] = (int64_t)tabs.size();
        const int Np = (int)ai.size();
        int f0 = -1, f1 = -1;
        for (int i = 0; i < Np; ++i) {
            const cd cm = -ai[i] * ah[i] * ih2s, c0 = ai[i] * (ah[i] + ah[i + 1]) * ih2s, cp = -ai[i] * ah[i + 1] * ih2s;
            tabs.push_back(cm);
            tabs.push_back(c0);
            tabs.push_back(cp);
            const bool plain = cm == cd(-ih2s, 0.0) && cp == cd(-ih2s, 0.0) && c0 == cd(2.0 * ih2s, 0.0);
            if (plain && f0 < 0) f0 = i;
            if (plain && f0 >= 0 && f1 < 0 && i == Np - 1) f1 = Np;
            if (!plain && f0 >= 0 && f1 < 0) f1 = i;
        }
        frange[a][0] = f0 < 0 ? 0 : f0;
        frange[a][1] = f0 < 0 ? 0 : f1;
    };
    stencil_axis(0, h->gx_int, h->gx_half);
    stencil_axis(1, h->gy_int, h->gy_half);
    stencil_axis(2, h->gz_int, h->gz_half);
    const int64_t stab0 = (int64_t)tabs.size();
    const int Ny = (int)h->N[1];
    for (auto& s : h->strips) {
        s.tab = (int64_t)tabs.size() - stab0;
        for (int c = 0; c < s.W; ++c) tabs.push_back(strip_alpha_at(h, s, 2 * c));
        for (int m = 0; m <= s.W; ++m) tabs.push_back(strip_alpha_at(h, s, 2 * m - 1));
    }
    // working-precision sweep tables: s_y, y-coupling -alpha_y(k-1/2)/h^2, strip s_x
    std::vector<cd> ctv;
    for (int k = 0; k < Ny; ++k) ctv.push_back(1.0 / h->gy_int[k]);
    const double ih2 = 1.0 / (h->h * h->h);
    for (int k = 0; k <= Ny; ++k) ctv.push_back(-h->gy_half[k] * ih2);
    for (auto& s : h->strips) {
        s.ctab = (int64_t)ctv.size();
        for (int c = 0; c < s.W; ++c) ctv.push_back(1.0 / tabs[stab0 + s.tab + c]);
    }
    h->ct_sz = (int64_t)ctv.size();   // s_z(z) (3-D strips)
    for (int z = 0; z < (int)h->N[2]; ++z) ctv.push_back(1.0 / h->gz_int[z]);
    if (h->d_ct) cudaFree(h->d_ct);
    h->d_ct = nullptr;
    CK(h, cudaMalloc(&h->d_ct, ctv.size() * h->esize));
    if (h->esize == sizeof(float2)) {
        std::vector<float2> f(ctv.size());
        for (size_t i = 0; i < ctv.size(); ++i) f[i] = make_float2((float)ctv[i].real(), (float)ctv[i].imag());
        CK(h, cudaMemcpy(h->d_ct, f.data(), f.size() * sizeof(float2), cudaMemcpyHostToDevice));
    } else {
        std::vector<double2> f(ctv.size());
        for (size_t i = 0; i < ctv.size(); ++i) f[i] = to_d2h(ctv[i]);
        CK(h, cudaMemcpy(h->d_ct, f.data(), f.size() * sizeof(double2), cudaMemcpyHostToDevice));
    }
    std::vector<double2> tab2(tabs.size());
    for (size_t i = 0; i < tabs.size(); ++i) tab2[i] = to_d2h(tabs[i]);
    if (h->d_tab) cudaFree(h->d_tab);
    if (h->d_strips) cudaFree(h->d_strips);
    if (h->d_ints) cudaFree(h->d_ints);
    h->d_tab = nullptr; h->d_strips = nullptr; h->d_ints = nullptr;
    CK(h, cudaMalloc(&h->d_tab, tab2.size() * sizeof(double2)));
    CK(h, cudaMalloc(&h->d_strips, h->strips.size() * sizeof(StripDev)));
    CK(h, cudaMalloc(&h->d_ints, (8 * h->P + 2 * h->P + Ny + 2 * h->G + h->sepmap.size()) * sizeof(int)));
    CK(h, cudaMemcpyAsync(h->d_tab, tab2.data(), tab2.size() * sizeof(double2), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->d_strips, h->strips.data(), h->strips.size() * sizeof(StripDev),
                          cudaMemcpyHostToDevice, h->stream));
    std::vector<int> ints;
    for (int p = 0; p < h->P; ++p) {   // chunk metadata of the finishing kernel
        int gs[2] = {-1, -1}, ra[2] = {0, 0}, rb[2] = {0, 0};
        for (int side = 0; side < 2; ++side) {
            const int q = side == 0 ? p - 1 : p;
            if (q < 0 || q >= h->P - 1 || h->G == 1 || h->sepmap[q] < 0) continue;
            const int gi = h->sepmap[q];
            gs[side] = gi;
            if (gi > 0) ra[side] = h->r1[h->gq0[gi] - 1];
            if (gi < h->G - 1) rb[side] = h->r1[h->gq1[gi]];
        }
        const int meta[8] = {h->r0[p], h->r1[p], gs[0], gs[1], ra[0], rb[0], ra[1], rb[1]};
        ints.insert(ints.end(), meta, meta + 8);
    }
    ints.insert(ints.end(), h->r0.begin(), h->r0.end());
    ints.insert(ints.end(), h->r1.begin(), h->r1.end());
    ints.insert(ints.end(), h->rowmap.begin(), h->rowmap.end());
    ints.insert(ints.end(), h->gq0.begin(), h->gq0.end());
    ints.insert(ints.end(), h->gq1.begin(), h->gq1.end());
    ints.insert(ints.end(), h->sepmap.begin(), h->sepmap.end());
    CK(h, cudaMemcpyAsync(h->d_ints, ints.data(), ints.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    if (h->d_icols) cudaFree(h->d_icols);
    h->d_icols = nullptr;
    CK(h, cudaMalloc(&h->d_icols, std::max<size_t>(h->icols.size(), 1) * sizeof(int)));
    if (!h->icols.empty())
        CK(h, cudaMemcpyAsync(h->d_icols, h->icols.data(), h->icols.size() * sizeof(int), cudaMemcpyHostToDevice,
                              h->stream));
    // Robin coefficients a/b per interface j and row (k^2 = omega^2 / c^2 as k_k2 forms it)
    if (h->d_rab) cudaFree(h->d_rab);
    h->d_rab = nullptr;
    if (h->transmission == HELM_TRANSMISSION_ROBIN && h->dim == 2) {
        std::vector<double2> rab((size_t)h->J * Ny, make_double2(0.0, 0.0));
        const int nx = (int)h->n[0], ny = (int)h->n[1], wo = h->w_outer;
        const double om2 = h->omega * h->omega;
        for (int j = 1; j < h->J; ++j) {
            const int col = h->beta[j] + 1;
            const int xi = std::min(std::max(col - wo, 0), nx - 1);
            for (int y = 0; y < Ny; ++y) {
                const int yi = std::min(std::max(y - wo, 0), ny - 1);
                const double cv = h->c[(size_t)yi * nx + xi];
                const double k = sqrt(om2 / (cv * cv));
                const cd a(1.0 / h->h, 0.5 * k), b(-1.0 / h->h, 0.5 * k);
                rab[(size_t)j * Ny + y] = to_d2h(a / b);
            }
        }
        CK(h, cudaMalloc(&h->d_rab, rab.size() * sizeof(double2)));
        CK(h, cudaMemcpyAsync(h->d_rab, rab.data(), rab.size() * sizeof(double2), cudaMemcpyHostToDevice, h->stream));
    }
    Geom& g = h->geom;
    g.dim = h->dim;
    g.Nx = (int)h->N[0];
    g.Ny = (int)h->N[1];
    g.Nz = (int)h->N[2];
    g.J = h->J;
    g.P = h->P;
    g.h = h->h;
    g.inv_h2 = 1.0 / (h->h * h->h);
    g.omega = h->omega;
    g.k2 = h->d_k2;
    int64_t o = 0;
    g.gx_int = h->d_tab + o; o += h->gx_int.size();
    g.gx_half = h->d_tab + o; o += h->gx_half.size();
    g.gy_int = h->d_tab + o; o += h->gy_int.size();
    g.gy_half = h->d_tab + o; o += h->gy_half.size();
    g.gz_int = h->d_tab + o; o += h->gz_int.size();
    g.gz_half = h->d_tab + o; o += h->gz_half.size();
    g.stab = h->d_tab + stab0;
    g.stc_x = h->d_tab + stc_off[0];
    g.stc_y = h->d_tab + stc_off[1];
    g.stc_z = h->d_tab + stc_off[2];
    g.fx0 = frange[0][0]; g.fx1 = frange[0][1];
    g.fy0 = frange[1][0]; g.fy1 = frange[1][1];
    g.fz0 = frange[2][0]; g.fz1 = frange[2][1];
    g.rab = h->d_rab;
    g.strips = h->d_strips;
    g.cmeta = reinterpret_cast<const int4*>(h->d_ints);
    g.r0 = h->d_ints + 8 * h->P;
    g.r1 = g.r0 + h->P;
    g.rowmap = g.r1 + h->P;
    g.G = h->G;
    g.gq0 = g.rowmap + Ny;
    g.gq1 = g.gq0 + h->G;
    g.sepmap = g.gq1 + h->G;
    if (h->counter_bytes != counter_bytes(h)) {
        if (h->d_counters) cudaFree(h->d_counters);
        h->d_counters = nullptr;
        h->counter_bytes = 0;
        CK(h, cudaMalloc(&h->d_counters, counter_bytes(h)));
        h->counter_bytes = counter_bytes(h);
    }
    CK(h, cudaMemsetAsync(h->d_counters, 0, h->counter_bytes, h->stream));
    g.ct = h->d_ct;
    g.ct_sy = 0;
    g.ct_cy = Ny;
    g.ct_sz = h->ct_sz;
    // rows of the sweep's z buffer: the longest chain one CTA runs (a chunk, a
    // separator group, or the level-2 system)
    h->zrows = std::max(h->G - 1, 1);
    for (int p = 0; p < h->P; ++p) h->zrows = std::max(h->zrows, h->r1[p] - h->r0[p]);
    for (int gi = 0; gi < h->G; ++gi) h->zrows = std::max(h->zrows, h->gq1[gi] - h->gq0[gi]);
    CK(h, cudaStreamSynchronize(h->stream));
    h->prepared = true;
    return HELM_OK;
}


// Output columns and transfer columns of strip j: the forward sweep keeps v^(j) on
// D^(j), the backward w^(j) on D~^(j); the transfer leaves strip j on its last two
// physical columns (forward, to the right neighbour) or its first two (backward).
void set_strip_io(const helm_dd* h, StripDev& s, int j) {
    s.olo[0] = h->beta[j] + 1;
    s.ohi[0] = h->beta[j + 1];
    s.olo[1] = j > 0 ? h->beta[j] + 2 : 0;
    s.ohi[1] = j < h->J - 1 ? h->beta[j + 1] + 1 : (int)h->N[0] - 1;   // D~^(J) ends at the grid's edge
    s.xc[1] = s.lpml + (s.hi - s.lo);
    s.xc[0] = s.xc[1] - 1;
    s.xc[2] = s.lpml;
    s.xc[3] = s.lpml + 1;
}

// Algorithm 1 on the strips of a 3-D grid: one dense block of n = W N_z unknowns per
// grid row y, X_k = S_k^{-1} stored for every row (slab3d.cu).
helm_status factor_slabs(helm_dd* h) {
    const int Ny = (int)h->N[1], Nz = (int)h->N[2];
    int64_t fac = 0;
    int nmax = 0, ldmax = 0;
    for (size_t jj = 0; jj < h->strips.size(); ++jj) {
        auto& s = h->strips[jj];
        set_strip_io(h, s, (int)jj);
        const int n = s.W * Nz;
        s.nj = 0;
        s.ld = (n + 3) & ~3;   // rows start 32-byte aligned, columns n.. zero
        s.bs = (int64_t)n * s.ld;
        s.fac = fac;
        s.red = 0;
        s.xf = 0;
        fac += (int64_t)Ny * s.bs;
        nmax = std::max(nmax, n);
        ldmax = std::max(ldmax, s.ld);
    }
    // dense blocks: up to 4096 unknowns in complex64 (the tensor-core factor and the wide strip
    // solve), 2048 in complex128
    const int nlim = h->esize == (int)sizeof(float2) ? 4096 : 2048;
    if (nmax > nlim)
        return fail(h, HELM_EINVAL, h->esize == (int)sizeof(float2)
                                        ? "a 3-D strip block has more than 4096 unknowns (W * N_z); use more strips"
                                        : "a complex128 3-D strip block has more than 2048 unknowns (W * N_z); use "
                                          "more strips or mixed precision");
    for (auto& p : h->d_pool) { if (p) cudaFree(p); p = nullptr; }
    h->factored = false;
    CK(h, cudaMalloc(&h->d_pool[0], (size_t)fac * h->esize));
    // s_x(c) s_z(z) per block entry, and the y-couplings
    std::vector<cd> sxz;
    h->slab_sxz_off.assign(h->strips.size(), 0);
    for (size_t jj = 0; jj < h->strips.size(); ++jj) {
        const auto& s = h->strips[jj];
        h->slab_sxz_off[jj] = (int64_t)sxz.size();
        for (int z = 0; z < Nz; ++z)
            for (int c = 0; c < s.W; ++c) sxz.push_back(1.0 / (strip_alpha_at(h, s, 2 * c) * h->gz_int[z]));
    }
    const double ih2 = 1.0 / (h->h * h->h);
    h->slab_cy.assign(Ny + 1, make_double2(0.0, 0.0));
    for (int k = 0; k <= Ny; ++k) h->slab_cy[k] = to_d2h(-h->gy_half[k] * ih2);
    if (h->d_slab_sxz) cudaFree(h->d_slab_sxz);
    h->d_slab_sxz = nullptr;
    CK(h, cudaMalloc(&h->d_slab_sxz, sxz.size() * h->esize));
    if (h->esize == sizeof(float2)) {
        std::vector<float2> f(sxz.size());
        for (size_t i = 0; i < sxz.size(); ++i) f[i] = make_float2((float)sxz[i].real(), (float)sxz[i].imag());
        CK(h, cudaMemcpy(h->d_slab_sxz, f.data(), f.size() * sizeof(float2), cudaMemcpyHostToDevice));
    } else {
        std::vector<double2> f(sxz.size());
        for (size_t i = 0; i < sxz.size(); ++i) f[i] = to_d2h(sxz[i]);
        CK(h, cudaMemcpy(h->d_slab_sxz, f.data(), f.size() * sizeof(double2), cudaMemcpyHostToDevice));
    }
    h->slab_ld = ldmax;
    CK(h, cudaMemcpyAsync(h->d_strips, h->strips.data(), h->strips.size() * sizeof(StripDev),
                          cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream));
    // scratch of the block inversions
    const size_t es = h->esize;
    const size_t mbytes = (size_t)ldmax * nmax * es, multb = (size_t)nmax * ldmax * es;
    const size_t ibytes = (size_t)(3 * nmax + 2) * sizeof(int);
    void* scratch = nullptr;
    CK(h, cudaMalloc(&scratch, mbytes + multb + ibytes));
    SlabScratch sc{};
    sc.M = scratch;
    sc.mult = (char*)scratch + mbytes;
    sc.ldm = ldmax;
    sc.perm = (int*)((char*)scratch + mbytes + multb);
    sc.pinv = sc.perm + nmax;
    sc.pivrow = sc.pinv + nmax;
    sc.bar = (unsigned*)(sc.pivrow + nmax);
    cudaError_t e = cudaSuccess;
    if (h->prec == HELM_PREC_MIXED) {
        // complex64: blocked Gauss-Jordan with tensor-core updates, up to 8 strips side by side
        const int ns_max = 8;
        void* tcs = nullptr;
        const size_t tcb = slab_factor_tc_scratch(nmax, std::min<int>(ns_max, (int)h->strips.size()));
        e = cudaMalloc(&tcs, tcb);
        for (size_t j0 = 0; j0 < h->strips.size() && e == cudaSuccess; j0 += ns_max) {
            const int ns = (int)std::min<size_t>(ns_max, h->strips.size() - j0);
            e = launch_slab_factor_tc(h->geom, h->strips.data() + j0, ns, h->d_pool[0], tcs, h->d_status, h->stream,
                                      &h->timer);
        }
        if (tcs) {
            cudaError_t e2 = cudaStreamSynchronize(h->stream);
            if (e == cudaSuccess) e = e2;
            cudaFree(tcs);
        }
    }
    for (size_t jj = 0; jj < h->strips.size() && e == cudaSuccess && h->prec != HELM_PREC_MIXED; ++jj)
        e = launch_slab_factor<double2>(h->geom, h->strips[jj], h->d_pool[0], sc, h->d_status, h->stream, &h->timer);
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(scratch);
    if (e != cudaSuccess) return fail_cuda(h, "3-D strip factor kernels", e);
    if (st == 7) {
        cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream);
        return fail(h, HELM_ETIMEOUT, "a bounded device wait in the 3-D strip factorisation gave up");
    }
    if (st != 0) return fail(h, HELM_ENUMERIC, "singular block in the strip factorisation");
    h->factored = true;
    return HELM_OK;
}

}  // namespace

// ============================================================== C ABI
extern "C" {

helm_status helm_dd_create(const helm_grid* g, const double* c, double omega, int w_outer, int w_sub, int J,
                           helm_prec prec, helm_dd** out) {
    if (out) *out = nullptr;
    if (!g || !c || !out) return HELM_EINVAL;
    if (g->dim != 2 && g->dim != 3) return HELM_EINVAL;
    if (!(g->h > 0) || !(omega > 0) || !isfinite(omega) || w_outer < 0 || J < 1) return HELM_EINVAL;
    if (J > 1 && w_sub < 1) return HELM_EINVAL;
    if (prec != HELM_PREC_FP64 && prec != HELM_PREC_MIXED) return HELM_EINVAL;
    for (int a = 0; a < g->dim; ++a)
        if (g->n[a] < 1 || g->n[a] > (1 << 20)) return HELM_EINVAL;
    const int64_t nz = g->dim == 3 ? g->n[2] : 1;
    const int64_t nint = g->n[0] * g->n[1] * nz;
    double cmax = 0.0;
    for (int64_t i = 0; i < nint; ++i) {
        if (!(c[i] > 0.0) || !isfinite(c[i])) return HELM_EINVAL;
        cmax = std::max(cmax, c[i]);
    }
    helm_dd* h = new helm_dd();
    h->dim = g->dim;
    for (int a = 0; a < 3; ++a) h->n[a] = (a < g->dim) ? g->n[a] : 1;
    for (int a = 0; a < 3; ++a) h->N[a] = (a < g->dim) ? h->n[a] + 2 * w_outer : 1;
    h->h = g->h;
    h->omega = omega;
    h->c_ref = cmax;
    h->w_outer = w_outer;
    h->w_sub = w_sub;
    h->J = J;
    h->prec = prec;
    h->esize = prec == HELM_PREC_MIXED ? sizeof(float2) : sizeof(double2);
    h->c.assign(c, c + nint);
    if (J > h->n[0]) { delete h; return HELM_EINVAL; }
    build_geometry(h);
    for (int j = 0; j < J; ++j) {
        const StripDev& s = h->strips[j];
        const int core = h->beta[j + 1] - h->beta[j];
        // strip blocks are dense W x W in shared memory: W <= 64
        if ((J > 1 && core < 2) || s.W > 64) { delete h; return HELM_EINVAL; }
    }
    *out = h;
    return HELM_OK;
}

helm_status helm_dd_set_pml_speed(helm_dd* h, double c_ref) {
    if (!h || !(c_ref > 0) || !isfinite(c_ref)) return HELM_EINVAL;
    if (h->factored) return fail(h, HELM_ESTATE, "set_pml_speed after factor");
    h->c_ref = c_ref;
    h->prepared = false;
    return HELM_OK;
}

helm_status helm_dd_set_chunks(helm_dd* h, int P) {
    if (!h || P < 0) return HELM_EINVAL;
    if (h->factored) return fail(h, HELM_ESTATE, "set_chunks after factor");
    if (P > 0 && 2 * P - 1 > h->N[1]) return fail(h, HELM_EINVAL, "too many chunks for the y extent");
    h->P_req = P;
    h->prepared = false;
    return HELM_OK;
}

helm_status helm_dd_set_sep_groups(helm_dd* h, int G) {
    if (!h || G < 0) return HELM_EINVAL;
    if (h->factored) return fail(h, HELM_ESTATE, "set_sep_groups after factor");
    h->G_req = G;
    h->prepared = false;
    return HELM_OK;
}

int helm_dd_sep_groups(const helm_dd* h) { return h && h->prepared ? h->G : 0; }

helm_status helm_dd_set_panel(helm_dd* h, int nrhs) {
    if (!h || nrhs < 0) return HELM_EINVAL;
    h->panel = nrhs;
    if (!h->factored) h->prepared = false;   // the built-in chunk count depends on it
    return HELM_OK;
}

int helm_dd_chunks(const helm_dd* h) { return h && h->prepared ? h->P : 0; }

helm_status helm_dd_set_sweep(helm_dd* h, helm_sweep mode) {
    if (!h || (mode != HELM_SWEEP_DOUBLE && mode != HELM_SWEEP_CONCURRENT)) return HELM_EINVAL;
    if (h->factored) return fail(h, HELM_ESTATE, "set_sweep after factor");
    if (mode == HELM_SWEEP_CONCURRENT && h->transmission != HELM_TRANSMISSION_PML)
        return fail(h, HELM_EINVAL, "concurrent sweeps use PML transmission");
    h->sweep = mode;
    h->prepared = false;
    return HELM_OK;
}

helm_status helm_dd_set_transmission(helm_dd* h, helm_transmission t) {
    if (!h || (t != HELM_TRANSMISSION_PML && t != HELM_TRANSMISSION_ROBIN)) return HELM_EINVAL;
    if (h->factored) return fail(h, HELM_ESTATE, "set_transmission after factor");
    if (t != HELM_TRANSMISSION_PML && h->sweep == HELM_SWEEP_CONCURRENT)
        return fail(h, HELM_EINVAL, "concurrent sweeps use PML transmission");
    h->transmission = t;
    build_geometry(h);
    h->prepared = false;
    return HELM_OK;
}

helm_status helm_dd_set_stream(helm_dd* h, void* stream) {
    if (!h) return HELM_EINVAL;
    h->stream = stream ? (cudaStream_t)stream : h->own_stream;   // null until first device use
    return HELM_OK;
}

helm_status helm_dd_set_timing(helm_dd* h, int enable) {
    if (!h) return HELM_EINVAL;
    if (h->stream) cudaStreamSynchronize(h->stream);
    h->timer.flush();
    if (enable) h->timer.reset();
    h->timer.enabled = enable != 0;
    return HELM_OK;
}

int helm_dd_kernel_stats(helm_dd* h, char (*names)[48], int64_t* launches, double* total_ms, int cap) {
    if (!h) return 0;
    if (h->stream) cudaStreamSynchronize(h->stream);
    h->timer.flush();
    const int n = (int)h->timer.names.size();
    for (int i = 0; i < n && i < cap; ++i) {
        if (names) { strncpy(names[i], h->timer.names[i].c_str(), 47); names[i][47] = 0; }
        if (launches) launches[i] = h->timer.counts[i];
        if (total_ms) total_ms[i] = h->timer.total_ms[i];
    }
    return n;
}

helm_status helm_dd_factor(helm_dd* h) {
    if (!h) return HELM_EINVAL;
    if (h->dim == 3 && h->transmission == HELM_TRANSMISSION_ROBIN)
        return fail(h, HELM_EINVAL, "Robin transmission is implemented for 2-D grids");
    if (h->dim == 3 && h->sweep == HELM_SWEEP_CONCURRENT)
        return fail(h, HELM_EINVAL, "concurrent sweeps are implemented for 2-D grids");
    helm_status ps = prepare_geom(h);
    if (ps != HELM_OK) return ps;
    if (h->dim == 3) return factor_slabs(h);
    const int Ny = (int)h->N[1];
    int64_t fac = 0, red = 0, xf = 0;
    for (size_t jj = 0; jj < h->strips.size(); ++jj) {
        auto& s = h->strips[jj];
        const int j = (int)jj;
        set_strip_io(h, s, j);
        s.nj = sweep_nj(s.W);
        s.ld = 4 * s.nj + 2;
        s.bs = (int64_t)s.W * s.ld;   // sweep layout; even, so blocks stay 16-byte aligned
        s.fac = fac;
        s.red = red;
        s.xf = xf;
        fac += (int64_t)Ny * s.bs;
        red += (int64_t)std::max(h->P - 1, 1) * s.bs;
        xf += (int64_t)Ny * 16 * spld(s.W);
        if (!strip_solve_fits(s, h->zrows, h->esize))
            return fail(h, HELM_EINVAL, "strip " + std::to_string(j) + " (" + std::to_string(s.W) +
                                            " columns) does not fit the strip solve's shared memory in " +
                                            (h->esize == sizeof(float2) ? "complex64" : "complex128") +
                                            " (complex128 strips hold at most about 50 columns): use more strips "
                                            "or mixed precision");
    }
    for (auto& p : h->d_pool) { if (p) cudaFree(p); p = nullptr; }
    h->factored = false;
    const size_t facb = (size_t)fac * h->esize, redb = (size_t)red * h->esize;
    CK(h, cudaMalloc(&h->d_pool[0], facb));
    CK(h, cudaMalloc(&h->d_pool[1], facb));
    CK(h, cudaMalloc(&h->d_pool[2], facb));
    CK(h, cudaMalloc(&h->d_pool[3], redb));
    CK(h, cudaMalloc(&h->d_pool[4], redb));
    CK(h, cudaMalloc(&h->d_pool[5], redb));
    if (h->G > 1) {
        for (int i = 6; i < 10; ++i) CK(h, cudaMalloc(&h->d_pool[i], redb));
        CK(h, cudaMalloc(&h->d_pool[10], (size_t)xf * h->esize));
        CK(h, cudaMalloc(&h->d_pool[11], redb));
        CK(h, cudaMalloc(&h->d_pool[12], redb));
    }
    CK(h, cudaMemcpyAsync(h->d_strips, h->strips.data(), h->strips.size() * sizeof(StripDev),
                          cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream));
    Geom& g = h->geom;
    cudaError_t e;
    if (h->prec == HELM_PREC_MIXED)
        e = launch_factor<float2>(g, h->Wmax, h->d_pool, h->d_status, h->stream, &h->timer);
    else
        e = launch_factor<double2>(g, h->Wmax, h->d_pool, h->d_status, h->stream, &h->timer);
    if (e != cudaSuccess) return fail_cuda(h, "factor kernels", e);
    int st = 0;
    CK(h, cudaMemcpyAsync(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (st != 0) return fail(h, HELM_ENUMERIC, "singular block in the strip factorisation");
    h->factored = true;
    return HELM_OK;
}

}  // extern "C"

namespace {

// out = A u (f == null) or f - A u, device fields [B][N]
helm_status dev_stencil(helm_dd* h, const double2* u, const double2* f, double2* out, int B) {
    CK(h, launch_stencil(h->geom, u, f, out, B, h->stream, &h->timer));
    return HELM_OK;
}

// Device error word: 7 = a bounded wait in a sweep kernel gave up.
helm_status check_device_status(helm_dd* h) {
    int st = 0;
    CK(h, cudaMemcpyAsync(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (st == 7) {
        cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream);
        cudaMemsetAsync(h->d_counters, 0, h->counter_bytes, h->stream);
        return fail(h, HELM_ETIMEOUT, "a bounded device wait in the sweep gave up");
    }
    return HELM_OK;
}

// Device buffers one preconditioner application works in.
struct PrecondBufs {
    double2* V;      // [B][N] forward-sweep field v
    double2* G;      // [B][N] residual g = f - A v
    void* Y;         // [J][B][Ny][ws] chain solutions of every strip, working precision (ws = work_stride)
    void* parts;     // per stream: separator right-hand-side parts, then level-2 contributions
    int* counters;   // [kMaxTiles][G+1] arrival counters, zero on entry
};
constexpr int kPrecondBufs = 4;

// Bytes of each PrecondBufs member (V, G, Y, parts) for B right-hand sides.
void precond_buf_bytes(const helm_dd* h, int B, size_t sz[kPrecondBufs]) {
    const int64_t NV = nvol(h);
    const int Ny = (int)h->N[1];
    sz[0] = (size_t)B * NV * sizeof(double2);
    sz[1] = sz[0];
    // concurrent sweeps keep three sets of chain solutions (upward, downward, corrections)
    // and one separator-parts buffer per stream
    sz[2] = (size_t)sweep_streams(h) * h->J * B * Ny * work_stride(h) * h->esize;
    sz[3] = (size_t)sweep_streams(h) * sweep_parts_total_bytes(h->P, B, work_stride(h), h->esize);
    if (h->dim == 3) {   // right-hand sides and two strip solutions, [B][Ny][slab_ld] each
        sz[2] = (size_t)3 * B * Ny * h->slab_ld * h->esize;
        sz[3] = 256;
    }
}

helm_status run_precond(helm_dd* h, const double2* in, double2* out, int B, const PrecondBufs& bf);
// The level-2 accumulators of a separator-parts buffer start at zero (each strip solve's
// level-2 CTA zeroes them again after reading them).
cudaError_t zero_acc2(helm_dd* h, void* parts, int B) {
    if (h->G <= 1) return cudaSuccess;
    const int ws = work_stride(h);
    return cudaMemsetAsync((char*)parts + sweep_parts_bytes(h->P, B, ws, h->esize), 0,
                           sweep_parts2_bytes(h->P, B, ws, h->esize), h->stream);
}
helm_status run_precond_slabs(helm_dd* h, const double2* in, double2* out, int B, const PrecondBufs& bf);
helm_status run_precond_concurrent(helm_dd* h, const double2* in, double2* out, int B, const PrecondBufs& bf);

// P applied to B device fields (Section 2.1): in -> out (distinct buffers).
helm_status dev_precond(helm_dd* h, const double2* in, double2* out, int B) {
    helm_status s;
    size_t sz[kPrecondBufs];
    precond_buf_bytes(h, B, sz);
    if ((s = ws_reserve(h, h->ws_V, sz[0])) != HELM_OK) return s;
    if ((s = ws_reserve(h, h->ws_G, sz[1])) != HELM_OK) return s;
    if ((s = ws_reserve(h, h->ws_Y, sz[2])) != HELM_OK) return s;
    if ((s = ws_reserve(h, h->ws_parts, sz[3])) != HELM_OK) return s;
    PrecondBufs bf{(double2*)h->ws_V.p, (double2*)h->ws_G.p, h->ws_Y.p, h->ws_parts.p, h->d_counters};
    return run_precond(h, in, out, B, bf);
}

// The work buffers a call reserves grow but never shrink; when the free device memory
// cannot hold `need` more bytes, drop them all so that the call's reservations start
// from a clean slate (a workspace kept for a wider earlier call would otherwise hold
// memory this call needs for others).
void release_if_short(helm_dd* h, size_t need) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { cudaGetLastError(); return; }
    if (fr >= need) return;
    cudaStreamSynchronize(h->stream);
    for (auto* w : {&h->ws_V, &h->ws_G, &h->ws_Y, &h->ws_parts, &h->ws_kry, &h->ws_small, &h->ws_red}) ws_free(*w);
}

// Right-hand sides per internal panel of a solve or gradient: as many as the free device
// memory holds, at most the handle's setting.  Per right-hand side a panel needs the
// FGMRES basis V_0..V_m, Z_0..Z_{m-1} and W (2m+2 fields), the preconditioner's
// forward field and residual (2 fields), `extra` fields of the caller and the
// strip chain solutions; the workspaces the handle already holds count as free.
int panel_width(helm_dd* h, int nrhs, int m, int extra) {
    if (h->panel > 0) nrhs = std::min(h->panel, nrhs);   // the caller's cap
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { cudaGetLastError(); return nrhs; }
    for (auto* w : {&h->ws_V, &h->ws_G, &h->ws_Y, &h->ws_parts, &h->ws_kry, &h->ws_small, &h->ws_grad}) fr += w->bytes;
    size_t sz[kPrecondBufs];
    precond_buf_bytes(h, 1, sz);
    const size_t field = (size_t)nvol(h) * sizeof(double2);
    const size_t per = (size_t)(2 * m + 2 + extra) * field + sz[0] + sz[1] + sz[2] + sz[3] + 4096;
    const size_t fit = (size_t)(0.85 * (double)fr) / per;
    const int Bp = (int)std::max<size_t>(1, std::min<size_t>((size_t)nrhs, fit));
    release_if_short(h, (size_t)Bp * per);
    return Bp;
}

// The double sweep itself on caller-provided buffers.
helm_status run_precond(helm_dd* h, const double2* in, double2* out, int B, const PrecondBufs& bf) {
    if (h->dim == 3) return run_precond_slabs(h, in, out, B, bf);
    if (h->sweep == HELM_SWEEP_CONCURRENT && h->J > 1) return run_precond_concurrent(h, in, out, B, bf);
    const int Ny = (int)h->N[1], Nx = (int)h->N[0];
    helm_status s;
    if (B > kMaxTiles) return fail(h, HELM_EINVAL, "too many right-hand sides in one call");
    double2* V = bf.V;
    double2* G = bf.G;
    const int ws = work_stride(h);
    const int64_t ystride = (int64_t)B * Ny * ws;
    const int J = h->J;
    const auto& beta = h->beta;
    const double ih2 = 1.0 / (h->h * h->h);
    const bool mixed = h->prec == HELM_PREC_MIXED;
    // strip j keeps its chain solution in its own slice: the next strip solve takes its
    // transfer from it, and the output columns of a whole sweep are written afterwards
    // in one launch
    auto ybuf = [&](int j) { return (char*)bf.Y + j * ystride * (int64_t)h->esize; };
    CK(h, zero_acc2(h, bf.parts, B));
    auto strip_solve = [&](int j, const SweepStep& sp) -> cudaError_t {
        SweepWork wk{ybuf(j), bf.parts, bf.counters, h->d_status, ws, B, h->zrows,
                     sp.prev >= 0 ? ybuf(sp.prev) : nullptr};
        const StripDev* pst = sp.prev >= 0 ? &h->strips[sp.prev] : nullptr;
        if (mixed)
            return launch_strip_solve<float2>(h->geom, j, h->strips[j], pst, sp, wk, h->d_pool, h->stream, &h->timer);
        return launch_strip_solve<double2>(h->geom, j, h->strips[j], pst, sp, wk, h->d_pool, h->stream, &h->timer);
    };
    const int kOutBatch = 8;    // strips per output launch
    // CTAs of an output launch beside the strip solves: the SMs a strip solve leaves free (one
    // CTA per chunk, one for the level-2 system when the separators are grouped); 56 when the
    // strip solve takes more than one wave anyway
    const int solve_ctas = h->P + (h->G > 1 ? 1 : 0);
    const int kOutCTAs = solve_ctas < h->nsm ? std::max(8, h->nsm - solve_ctas) : 56;
    // Output columns of strips jlo .. jlo+n-1, once their solves are done: on the side
    // stream, so that they run on the SMs the strip solves leave idle; join() makes the
    // main stream wait for every output pass issued so far.
    // Passes issued while strip solves still follow run on a third of the SMs (the strip
    // solves take about two thirds); the last pass of a sweep runs on the whole GPU.
    auto outputs = [&](int dir, int jlo, int n, double2* dst, const double2* base, bool last) -> cudaError_t {
        if (n <= 0) return cudaSuccess;
        OutArgs O{h->geom, dir, jlo, n, bf.Y, ystride, ws, B, B > 1 ? 4 : 1, dst, base, last ? 0 : kOutCTAs};
        cudaError_t e = cudaEventRecord(h->ev_main, h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side, h->ev_main, 0);
        if (e != cudaSuccess) return e;
        if (mixed) return launch_outputs<float2>(O, h->d_pool, h->side, &h->timer);
        return launch_outputs<double2>(O, h->d_pool, h->side, &h->timer);
    };
    auto join = [&]() -> cudaError_t {
        cudaError_t e = cudaEventRecord(h->ev_side, h->side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_side, 0);
        return e;
    };

    // forward sweep j = 1..J (Eq. solve_upward): A^(j) v^(j) = 1_{D^(j)} f - 2 delta(x-b_j) d_x v^(j-1),
    // the transfer on the first two columns of strip j taken from the solve of strip j-1
    for (int j = 0; j < J; ++j) {
        SweepStep sp{};
        sp.src = in;
        sp.mlo = beta[j] + 1;
        sp.mhi = beta[j + 1];
        sp.prev = j > 0 ? j - 1 : -1;
        sp.pdir = 0;
        sp.t0 = beta[j];
        sp.tcoef = -ih2;
        if (h->d_rab && j > 0) {   // Robin data d_x v + ik v at l^(j) (Section 4.4)
            sp.tcoef = ih2;
            sp.rbk = h->d_rab + (int64_t)j * Ny;
            sp.rb_in = 1;
        }
        CK(h, strip_solve(j, sp));
        if ((j + 1) % kOutBatch == 0 || j == J - 1)
            CK(h, outputs(0, j + 1 - ((j % kOutBatch) + 1), (j % kOutBatch) + 1, (J == 1) ? out : V, nullptr,
                          j == J - 1));
    }
    CK(h, join());
    if (J == 1) return HELM_OK;
    // residual g = f - A v
    if ((s = dev_stencil(h, V, in, G, B)) != HELM_OK) return s;
    // backward sweep j = J-1..1 (Eq. solve_downward), w^(J) = 0, out = v + w on D~^(j),
    // the transfer on columns beta_{j+1}+1, +2 taken from the solve of strip j+1
    for (int j = J - 2; j >= 0; --j) {
        SweepStep sp{};
        sp.src = G;
        sp.mlo = j > 0 ? beta[j] + 2 : 0;
        sp.mhi = beta[j + 1] + 1;
        sp.prev = (j + 1 <= J - 2) ? j + 1 : -1;
        sp.pdir = 1;
        sp.t0 = beta[j + 1] + 1;
        sp.tcoef = ih2;
        if (h->d_rab && sp.prev >= 0) {   // Robin data -d_x w + ik w at r^(j)
            sp.rbk = h->d_rab + (int64_t)(j + 1) * Ny;
            sp.rb_in = 0;
        }
        CK(h, strip_solve(j, sp));
        const int done = J - 1 - j;   // strips solved so far in this sweep: j .. J-2
        if (done % kOutBatch == 0 || j == 0) CK(h, outputs(1, j, (done - 1) % kOutBatch + 1, out, V, j == 0));
    }
    CK(h, join());
    // D~^(J) keeps v (w = 0 there)
    CK(h, launch_copy_cols(V, out, B, Nx, Ny, (int)h->N[2], beta[J - 1] + 2, Nx - 1, h->stream, &h->timer));
    return HELM_OK;
}

// The double sweep on the strips of a 3-D grid (same steps as run_precond; each strip
// solve is the block substitution of slab3d.cu, its output written right after it).
helm_status run_precond_slabs(helm_dd* h, const double2* in, double2* out, int B, const PrecondBufs& bf) {
    const int Ny = (int)h->N[1], Nx = (int)h->N[0], Nz = (int)h->N[2];
    const int J = h->J, ld = h->slab_ld;
    const auto& beta = h->beta;
    const double ih2 = 1.0 / (h->h * h->h);
    const bool mixed = h->prec == HELM_PREC_MIXED;
    const size_t vb = (size_t)B * Ny * ld * h->esize;
    char* rbuf = (char*)bf.Y;
    char* ybuf[2] = {rbuf + vb, rbuf + 2 * vb};
    double2* V = bf.V;
    helm_status s;
    auto solve = [&](int j, const SweepStep& sp, int slot) -> cudaError_t {
        SlabWork wk{rbuf, ybuf[slot], sp.prev >= 0 ? ybuf[slot ^ 1] : nullptr,
                    (const char*)h->d_slab_sxz + h->slab_sxz_off[j] * (int64_t)h->esize, h->ct_sz,
                    h->slab_cy.data(), ld, B, (unsigned*)bf.counters, h->d_status};
        const StripDev* pst = sp.prev >= 0 ? &h->strips[sp.prev] : nullptr;
        if (mixed) return launch_slab_solve<float2>(h->geom, h->strips[j], pst, sp, wk, h->d_pool[0], h->stream, &h->timer);
        return launch_slab_solve<double2>(h->geom, h->strips[j], pst, sp, wk, h->d_pool[0], h->stream, &h->timer);
    };
    auto emit = [&](int j, int dir, int slot, double2* dst, const double2* base) -> cudaError_t {
        if (mixed) return launch_slab_out<float2>(h->geom, h->strips[j], dir, ybuf[slot], ld, dst, base, B, h->stream, &h->timer);
        return launch_slab_out<double2>(h->geom, h->strips[j], dir, ybuf[slot], ld, dst, base, B, h->stream, &h->timer);
    };
    for (int j = 0; j < J; ++j) {   // forward sweep (Eq. solve_upward)
        SweepStep sp{};
        sp.src = in;
        sp.mlo = beta[j] + 1;
        sp.mhi = beta[j + 1];
        sp.prev = j > 0 ? j - 1 : -1;
        sp.pdir = 0;
        sp.t0 = beta[j];
        sp.tcoef = -ih2;
        CK(h, solve(j, sp, j & 1));
        CK(h, emit(j, 0, j & 1, J == 1 ? out : V, nullptr));
    }
    if (J == 1) return HELM_OK;
    if ((s = dev_stencil(h, V, in, bf.G, B)) != HELM_OK) return s;
    for (int j = J - 2; j >= 0; --j) {   // backward sweep (Eq. solve_downward), w^(J) = 0
        SweepStep sp{};
        sp.src = bf.G;
        sp.mlo = j > 0 ? beta[j] + 2 : 0;
        sp.mhi = beta[j + 1] + 1;
        sp.prev = (j + 1 <= J - 2) ? j + 1 : -1;
        sp.pdir = 1;
        sp.t0 = beta[j + 1] + 1;
        sp.tcoef = ih2;
        const int slot = (J - 2 - j) & 1;
        CK(h, solve(j, sp, slot));
        CK(h, emit(j, 1, slot, out, V));
    }
    CK(h, launch_copy_cols(V, out, B, Nx, Ny, Nz, beta[J - 1] + 2, Nx - 1, h->stream, &h->timer));
    return HELM_OK;
}

// The upward and downward sequences performed simultaneously (Section 1.2 "Results";
// Section 3.1), PML transfers.  Three streams run strip solves side by side:
//   upward (the handle's stream):  v^(j), j = 1..J, f on D^(j) + the transfer from v^(j-1);
//   downward (cstream[0]):         y^(j), j = J..2, f on D~^(j) + the transfer from y^(j+1);
//   corrections (cstream[1]):      s^(j), j = 1..J-1, f on the overlap column beta_j+1 +
//                                  the transfer from y^(j+1), each once y^(j+1) is done.
// Strip j's total field, A^(j) u^(j) = f on its physical columns + both transfers, is
// v^(j) + s^(j) by linearity (u^(J) = v^(J)); out = u^(j) on D^(j).  Each stream has
// its own separator-parts buffer and arrival counters.
helm_status run_precond_concurrent(helm_dd* h, const double2* in, double2* out, int B, const PrecondBufs& bf) {
    const int Ny = (int)h->N[1], Nx = (int)h->N[0];
    if (B > kMaxTiles) return fail(h, HELM_EINVAL, "too many right-hand sides in one call");
    double2* V = bf.V;
    const int ws = work_stride(h);
    const int64_t ystride = (int64_t)B * Ny * ws;
    const int J = h->J;
    const auto& beta = h->beta;
    const double ih2 = 1.0 / (h->h * h->h);
    const bool mixed = h->prec == HELM_PREC_MIXED;
    const size_t es = h->esize;
    char* Yset[3] = {(char*)bf.Y, (char*)bf.Y + (size_t)J * ystride * es, (char*)bf.Y + (size_t)2 * J * ystride * es};
    const size_t psz = sweep_parts_total_bytes(h->P, B, ws, es);
    void* parts[3] = {bf.parts, (char*)bf.parts + psz, (char*)bf.parts + 2 * psz};
    for (void* pp : parts) CK(h, zero_acc2(h, pp, B));
    const size_t cset = counter_set_bytes(h) / sizeof(int);
    int* ctr[3] = {bf.counters, bf.counters + cset, bf.counters + 2 * cset};
    cudaStream_t st[3] = {h->stream, h->cstream[0], h->cstream[1]};
    auto ybuf = [&](int set, int j) { return Yset[set] + (size_t)j * ystride * es; };
    // set: 0 upward, 1 downward, 2 corrections; the transfer comes from set `pset`
    auto strip_solve = [&](int set, int j, const SweepStep& sp, int pset) -> cudaError_t {
        SweepWork wk{ybuf(set, j), parts[set], ctr[set], h->d_status, ws, B, h->zrows,
                     sp.prev >= 0 ? ybuf(pset, sp.prev) : nullptr};
        wk.pdl = false;   // a pre-launched successor would hold SMs the other streams need
        const StripDev* pst = sp.prev >= 0 ? &h->strips[sp.prev] : nullptr;
        if (mixed)
            return launch_strip_solve<float2>(h->geom, j, h->strips[j], pst, sp, wk, h->d_pool, st[set], &h->timer);
        return launch_strip_solve<double2>(h->geom, j, h->strips[j], pst, sp, wk, h->d_pool, st[set], &h->timer);
    };
    auto outputs = [&](int set, int jlo, int n, double2* dst, const double2* base, int maxcta) -> cudaError_t {
        if (n <= 0) return cudaSuccess;
        OutArgs O{h->geom, 0, jlo, n, Yset[set], ystride, ws, B, B > 1 ? 4 : 1, dst, base, maxcta};
        if (mixed) return launch_outputs<float2>(O, h->d_pool, h->side, &h->timer);
        return launch_outputs<double2>(O, h->d_pool, h->side, &h->timer);
    };
    cudaEvent_t ev_fork = h->cev[0], ev_y = h->cev[1], ev_down = h->cev[2], ev_corr = h->cev[3];
    // fork: the other two streams start once the input is ready on the handle's stream
    CK(h, cudaEventRecord(ev_fork, st[0]));
    CK(h, cudaStreamWaitEvent(st[1], ev_fork, 0));
    CK(h, cudaStreamWaitEvent(st[2], ev_fork, 0));
    const int kOutBatch = 8;
    // Issue the three sequences interleaved in time order, so that each stream's next
    // launch is queued while the others run.
    for (int t = 0; t < J; ++t) {
        {   // upward: v^(t)
            const int j = t;
            SweepStep sp{};
            sp.src = in;
            sp.mlo = beta[j] + 1;
            sp.mhi = beta[j + 1];
            sp.prev = j > 0 ? j - 1 : -1;
            sp.pdir = 0;
            sp.t0 = beta[j];
            sp.tcoef = -ih2;
            CK(h, strip_solve(0, j, sp, 0));
            if ((j + 1) % kOutBatch == 0 || j == J - 1) {   // v on D^(j), beside the solves
                CK(h, cudaEventRecord(h->ev_main, st[0]));
                CK(h, cudaStreamWaitEvent(h->side, h->ev_main, 0));
                const int n = (j % kOutBatch) + 1;
                CK(h, outputs(0, j + 1 - n, n, V, nullptr, j == J - 1 ? 0 : 56));
            }
        }
        const int j = J - 1 - t;   // downward: y^(j), j = J-1 .. 1; then the correction s^(j-1)
        if (j >= 1) {
            SweepStep sp{};
            sp.src = in;
            sp.mlo = beta[j] + 2;
            sp.mhi = j < J - 1 ? beta[j + 1] + 1 : Nx - 1;
            sp.prev = j < J - 1 ? j + 1 : -1;
            sp.pdir = 1;
            sp.t0 = beta[j + 1] + 1;
            sp.tcoef = ih2;
            CK(h, strip_solve(1, j, sp, 1));
            CK(h, cudaEventRecord(ev_y, st[1]));
            CK(h, cudaStreamWaitEvent(st[2], ev_y, 0));
            SweepStep sc{};
            sc.src = in;
            sc.mlo = beta[j] + 1;   // strip j-1's overlap column
            sc.mhi = beta[j] + 1;
            sc.prev = j;
            sc.pdir = 1;
            sc.t0 = beta[j] + 1;
            sc.tcoef = ih2;
            CK(h, strip_solve(2, j - 1, sc, 1));
        }
    }
    // out = v + s on D^(j), j < J-1 (after the v outputs on the side stream and every
    // correction), and v on D^(J)
    CK(h, cudaEventRecord(ev_corr, st[2]));
    CK(h, cudaStreamWaitEvent(h->side, ev_corr, 0));
    CK(h, outputs(2, 0, J - 1, out, V, 0));
    CK(h, cudaEventRecord(ev_down, st[1]));
    CK(h, cudaStreamWaitEvent(st[0], ev_down, 0));
    CK(h, cudaEventRecord(h->ev_side, h->side));
    CK(h, cudaStreamWaitEvent(st[0], h->ev_side, 0));
    CK(h, launch_copy_cols(V, out, B, Nx, Ny, (int)h->N[2], beta[J - 1] + 1, Nx - 1, st[0], &h->timer));
    return HELM_OK;
}

struct IoField {
    const double* user_in = nullptr;
    double* user_out = nullptr;
    bool dev_in = false, dev_out = false;
};

}  // namespace

extern "C" {

helm_status helm_dd_apply_precond(helm_dd* h, const double* in, double* out, int nrhs) {
    if (!h || !in || !out || nrhs < 1) return HELM_EINVAL;
    if (!h->factored) return fail(h, HELM_ESTATE, "apply_precond before factor");
    const size_t bytes = (size_t)nrhs * nvol(h) * sizeof(double2);
    const bool din = is_device_ptr(in), dout = is_device_ptr(out);
    if ((din && misaligned16(in)) || (dout && misaligned16(out)))
        return fail(h, HELM_EINVAL, "device fields must be 16-byte aligned (complex128)");
    helm_status s;
    const double2* dinp = (const double2*)in;
    double2* doutp = (double2*)out;
    if (!din) {
        if ((s = ws_reserve(h, h->ws_io_in, bytes)) != HELM_OK) return s;
        CK(h, cudaMemcpyAsync(h->ws_io_in.p, in, bytes, cudaMemcpyHostToDevice, h->stream));
        dinp = (const double2*)h->ws_io_in.p;
    }
    if (!dout || (const void*)doutp == (const void*)dinp) {
        if ((s = ws_reserve(h, h->ws_io_out, bytes)) != HELM_OK) return s;
        doutp = (double2*)h->ws_io_out.p;
    }
    if ((s = dev_precond(h, dinp, doutp, nrhs)) != HELM_OK) return s;
    if ((s = check_device_status(h)) != HELM_OK) return s;
    if (!dout) CK(h, cudaMemcpyAsync(out, doutp, bytes, cudaMemcpyDeviceToHost, h->stream));
    else if ((void*)doutp != (void*)out)
        CK(h, cudaMemcpyAsync(out, doutp, bytes, cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return HELM_OK;
}

helm_status helm_dd_matvec(helm_dd* h, const double* in, double* out, int nrhs) {
    if (!h || !in || !out || nrhs < 1) return HELM_EINVAL;
    if (!h->prepared) {
        helm_status ps = prepare_geom(h);
        if (ps != HELM_OK) return ps;
    }
    const size_t bytes = (size_t)nrhs * nvol(h) * sizeof(double2);
    const bool din = is_device_ptr(in), dout = is_device_ptr(out);
    if ((din && misaligned16(in)) || (dout && misaligned16(out)))
        return fail(h, HELM_EINVAL, "device fields must be 16-byte aligned (complex128)");
    helm_status s;
    const double2* dinp = (const double2*)in;
    double2* doutp = (double2*)out;
    if (!din) {
        if ((s = ws_reserve(h, h->ws_io_in, bytes)) != HELM_OK) return s;
        CK(h, cudaMemcpyAsync(h->ws_io_in.p, in, bytes, cudaMemcpyHostToDevice, h->stream));
        dinp = (const double2*)h->ws_io_in.p;
    }
    if (!dout) {
        if ((s = ws_reserve(h, h->ws_io_out, bytes)) != HELM_OK) return s;
        doutp = (double2*)h->ws_io_out.p;
    }
    if ((s = dev_stencil(h, dinp, nullptr, doutp, nrhs)) != HELM_OK) return s;
    if (!dout) CK(h, cudaMemcpyAsync(out, doutp, bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return HELM_OK;
}

}  // extern "C"

namespace {

// The operator a GMRES run works on, over vectors of n entries per right-hand side:
// residual(x, f, out, B) writes out = f - M x (out = M x when f is null); precond(v, z, B)
// writes z = P v, or is empty for plain GMRES (no preconditioner inside the operator's
// Krylov loop, x += V y).
struct KrylovOp {
    int64_t n = 0;
    std::function<helm_status(const double2*, const double2*, double2*, int)> residual;
    std::function<helm_status(const double2*, double2*, int)> precond;
    // stop on the Givens estimate without forming the final residual (the caller checks
    // the true residual itself); for operators whose every application is expensive
    bool trust_estimate = false;
};

// GMRES(m) on op (Section 2.3; Algorithm 5), batched over B columns with per-column
// masks; with a preconditioner it is right-preconditioned flexible GMRES (Z_i = P V_i
// stored, x += Z y), which admits the complex64 preconditioner.  Classical Gram-Schmidt
// with reorthogonalisation (CGS2) in FP64 on the device; Hessenberg, Givens rotations and
// the small triangular solve on the host.
helm_status dev_gmres(helm_dd* h, const KrylovOp& op, const double2* F, double2* U, int B, double tol, int m,
                      int maxit, std::vector<int>& iters, std::vector<double>& relres,
                      const std::vector<double>* tol_per = nullptr) {
    const int64_t NV = op.n;
    // relative tolerance of column b (one for all, or one per column)
    auto tolb = [&](int b) { return tol_per ? (*tol_per)[b] : tol; };
    const size_t vb = (size_t)B * NV * sizeof(double2);
    const bool flex = (bool)op.precond;
    helm_status s;
    // Krylov storage: V_0..V_m, Z_0..Z_{m-1} (flexible only), W
    if ((s = ws_reserve(h, h->ws_kry, (size_t)(flex ? 2 * m + 2 : m + 2) * vb)) != HELM_OK) return s;
    const int nblk = 304;
    const size_t small = (size_t)B * (m + 2) * nblk * sizeof(double2) + (size_t)4 * B * (m + 2) * sizeof(double2);
    if ((s = ws_reserve(h, h->ws_small, small)) != HELM_OK) return s;
    double2* V = (double2*)h->ws_kry.p;
    const int64_t vs = (int64_t)B * NV;   // stride between Krylov vectors (elements)
    double2* Z = flex ? V + (int64_t)(m + 1) * vs : V;
    double2* Wv = flex ? Z + (int64_t)m * vs : V + (int64_t)(m + 1) * vs;
    double2* partial = (double2*)h->ws_small.p;
    double2* dres = partial + (size_t)B * (m + 2) * nblk;
    double2* dcoef = dres + (size_t)B * (m + 2);
    double* dscale = (double*)(dcoef + (size_t)B * (m + 2));
    std::vector<double2> hres(B * (m + 2)), hcoef(B * (m + 2));
    std::vector<double> hscale(B);

    auto norms = [&](const double2* X, std::vector<double>& nrm) -> helm_status {
        CK(h, launch_multidot(X, 0, X, 1, B, NV, partial, nblk, dres, h->stream, &h->timer));
        CK(h, cudaMemcpyAsync(hres.data(), dres, B * sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        nrm.resize(B);
        for (int b = 0; b < B; ++b) nrm[b] = sqrt(std::max(hres[b].x, 0.0));
        return HELM_OK;
    };

    std::vector<double> bnorm;
    if ((s = norms(F, bnorm)) != HELM_OK) return s;
    for (int b = 0; b < B; ++b)
        if (!isfinite(bnorm[b])) return fail(h, HELM_ENUMERIC, "non-finite right-hand side");
    CK(h, cudaMemsetAsync(U, 0, vb, h->stream));
    iters.assign(B, 0);
    relres.assign(B, 0.0);
    std::vector<char> conv(B, 0);
    std::vector<cd> H((size_t)B * (m + 1) * m), g((size_t)B * (m + 1)), sn((size_t)B * m);
    std::vector<double> cs((size_t)B * m);
    std::vector<int> kend(B);
    std::vector<char> active(B);
    std::vector<double> beta;
    std::vector<double> last_est(B, 0.0);
    int guard = 0;
    bool first = true;
    while (true) {
        // r = f - M x into V_0 (r = f for the first cycle, where x = 0)
        if (first) CK(h, cudaMemcpyAsync(V, F, vb, cudaMemcpyDeviceToDevice, h->stream));
        else if ((s = op.residual(U, F, V, B)) != HELM_OK) return s;
        first = false;
        if ((s = norms(V, beta)) != HELM_OK) return s;
        bool any = false;
        for (int b = 0; b < B; ++b) {
            if (!isfinite(beta[b])) return fail(h, HELM_ENUMERIC, "non-finite residual norm");
            relres[b] = bnorm[b] > 0 ? beta[b] / bnorm[b] : 0.0;
            if (bnorm[b] == 0.0 || beta[b] <= tolb(b) * bnorm[b]) conv[b] = 1;
            active[b] = !conv[b] && iters[b] < maxit;
            any = any || active[b];
            hscale[b] = active[b] ? 1.0 / beta[b] : 0.0;
            kend[b] = 0;
            for (int i = 0; i <= m; ++i) g[(size_t)b * (m + 1) + i] = 0.0;
            g[(size_t)b * (m + 1)] = beta[b];
        }
        if (!any || ++guard > 100000) break;
        CK(h, cudaMemcpyAsync(dscale, hscale.data(), B * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CK(h, launch_scale(V, V, dscale, B, NV, h->stream, &h->timer));
        for (int i = 0; i < m; ++i) {
            double2* Vi = V + (int64_t)i * vs;
            double2* Zi = Z + (int64_t)i * vs;
            if (flex && (s = op.precond(Vi, Zi, B)) != HELM_OK) return s;
            if ((s = op.residual(Zi, nullptr, Wv, B)) != HELM_OK) return s;
            // CGS2
            std::vector<cd> hcol((size_t)B * (i + 1), 0.0);
            for (int pass = 0; pass < 2; ++pass) {
                CK(h, launch_multidot(V, vs, Wv, i + 1, B, NV, partial, nblk, dres, h->stream, &h->timer));
                CK(h, cudaMemcpyAsync(hres.data(), dres, (size_t)B * (i + 1) * sizeof(double2),
                                      cudaMemcpyDeviceToHost, h->stream));
                CK(h, cudaStreamSynchronize(h->stream));
                for (int b = 0; b < B; ++b)
                    for (int k = 0; k <= i; ++k) {
                        const double2 v = hres[(size_t)b * (i + 1) + k];
                        const cd hv = active[b] ? cd(v.x, v.y) : cd(0.0);
                        hcol[(size_t)b * (i + 1) + k] += hv;
                        hcoef[(size_t)b * (i + 1) + k] = make_double2(-hv.real(), -hv.imag());
                    }
                CK(h, cudaMemcpyAsync(dcoef, hcoef.data(), (size_t)B * (i + 1) * sizeof(double2),
                                      cudaMemcpyHostToDevice, h->stream));
                CK(h, launch_multi_axpy(Wv, V, vs, dcoef, i + 1, B, NV, h->stream, &h->timer));
            }
            std::vector<double> hn;
            if ((s = norms(Wv, hn)) != HELM_OK) return s;
            bool still = false;
            for (int b = 0; b < B; ++b) {
                if (!active[b]) { hscale[b] = 0.0; continue; }
                if (!isfinite(hn[b])) return fail(h, HELM_ENUMERIC, "non-finite Arnoldi norm");
                cd* Hb = &H[(size_t)b * (m + 1) * m];
                auto Hc = [&](int r, int c) -> cd& { return Hb[(size_t)c * (m + 1) + r]; };
                for (int k = 0; k <= i; ++k) Hc(k, i) = hcol[(size_t)b * (i + 1) + k];
                Hc(i + 1, i) = hn[b];
                double* csb = &cs[(size_t)b * m];
                cd* snb = &sn[(size_t)b * m];
                for (int k = 0; k < i; ++k) {
                    const cd t = csb[k] * Hc(k, i) + snb[k] * Hc(k + 1, i);
                    Hc(k + 1, i) = -std::conj(snb[k]) * Hc(k, i) + csb[k] * Hc(k + 1, i);
                    Hc(k, i) = t;
                }
                const cd a = Hc(i, i);
                const double bb = hn[b];
                const double rho = hypot(std::abs(a), bb);
                if (std::abs(a) == 0.0) {
                    csb[i] = 0.0;
                    snb[i] = 1.0;
                    Hc(i, i) = bb;
                } else {
                    csb[i] = std::abs(a) / rho;
                    snb[i] = (a / std::abs(a)) * bb / rho;
                    Hc(i, i) = (a / std::abs(a)) * rho;
                }
                Hc(i + 1, i) = 0.0;
                cd* gb = &g[(size_t)b * (m + 1)];
                gb[i + 1] = -std::conj(snb[i]) * gb[i];
                gb[i] = csb[i] * gb[i];
                iters[b] += 1;
                kend[b] = i + 1;
                const double est = std::abs(gb[i + 1]);
                last_est[b] = est;
                if (est <= tolb(b) * bnorm[b] || iters[b] >= maxit || hn[b] == 0.0) active[b] = 0;
                hscale[b] = (active[b] && hn[b] > 0) ? 1.0 / hn[b] : 0.0;
                still = still || active[b];
            }
            if (!still || i == m - 1) break;
            CK(h, cudaMemcpyAsync(dscale, hscale.data(), B * sizeof(double), cudaMemcpyHostToDevice, h->stream));
            CK(h, launch_scale(V + (int64_t)(i + 1) * vs, Wv, dscale, B, NV, h->stream, &h->timer));
        }
        // x += Z y,  H y = g (upper triangular, per column)
        int kmax = 0;
        for (int b = 0; b < B; ++b) kmax = std::max(kmax, kend[b]);
        for (int b = 0; b < B; ++b) {
            cd* Hb = &H[(size_t)b * (m + 1) * m];
            auto Hc = [&](int r, int c) -> cd& { return Hb[(size_t)c * (m + 1) + r]; };
            std::vector<cd> y(kend[b]);
            for (int k = kend[b] - 1; k >= 0; --k) {
                cd acc = g[(size_t)b * (m + 1) + k];
                for (int l = k + 1; l < kend[b]; ++l) acc -= Hc(k, l) * y[l];
                y[k] = acc / Hc(k, k);
            }
            for (int k = 0; k < kmax; ++k) {
                const cd v = k < kend[b] ? y[k] : cd(0.0);
                hcoef[(size_t)b * kmax + k] = make_double2(v.real(), v.imag());
            }
        }
        if (kmax > 0) {
            CK(h, cudaMemcpyAsync(dcoef, hcoef.data(), (size_t)B * kmax * sizeof(double2), cudaMemcpyHostToDevice,
                                  h->stream));
            CK(h, launch_multi_axpy(U, Z, vs, dcoef, kmax, B, NV, h->stream, &h->timer));
        }
        if (op.trust_estimate) {   // done when every column met its tolerance or maxit by the estimate
            bool done = true;
            for (int b = 0; b < B; ++b) {
                if (conv[b]) continue;
                if (kend[b] > 0) relres[b] = bnorm[b] > 0 ? last_est[b] / bnorm[b] : 0.0;
                if (!(relres[b] <= tolb(b)) && iters[b] < maxit) done = false;
            }
            if (done) {
                bool allconv = true;
                for (int b = 0; b < B; ++b) allconv = allconv && relres[b] <= tolb(b);
                return allconv ? HELM_OK : fail(h, HELM_ENOTCONV, "GMRES reached maxit before the tolerance");
            }
        }
    }
    // final true residual
    if ((s = op.residual(U, F, Wv, B)) != HELM_OK) return s;
    std::vector<double> rn;
    if ((s = norms(Wv, rn)) != HELM_OK) return s;
    bool allconv = true;
    for (int b = 0; b < B; ++b) {
        relres[b] = bnorm[b] > 0 ? rn[b] / bnorm[b] : 0.0;
        if (!(relres[b] <= tolb(b))) allconv = false;
    }
    return allconv ? HELM_OK : fail(h, HELM_ENOTCONV, "GMRES reached maxit before the tolerance");
}

// Flexible GMRES in the full space (Algorithm 5 in its full-space form): A P v = f,
// u = P v, over all padded unknowns.
helm_status dev_fgmres(helm_dd* h, const double2* F, double2* U, int B, double tol, int m, int maxit,
                       std::vector<int>& iters, std::vector<double>& relres) {
    KrylovOp op;
    op.n = nvol(h);
    op.residual = [h](const double2* x, const double2* f, double2* out, int nb) {
        return dev_stencil(h, x, f, out, nb);
    };
    op.precond = [h](const double2* v, double2* z, int nb) { return dev_precond(h, v, z, nb); };
    return dev_gmres(h, op, F, U, B, tol, m, maxit, iters, relres);
}


// ------------------------------------------------------------------ reduced space
// Section 2.3 ("Algorithm"), Algorithms 2-5: GMRES restricted to the 2(J-1) interface
// lines beta_j+1, beta_j+2 (j = 1..J-1).  A reduced vector holds B fields of N_z N_y rows
// of L = 2(J-1) values: entry (b, z, y, i) is column icols[i] of row (z, y) of field b.

int64_t nred(const helm_dd* h) { return h->N[2] * h->N[1] * (int64_t)h->icols.size(); }

// Algorithm 2, the strip solves (Eq. reduce_compute_ut): u~^(j) from f restricted to
// D~^(j) = beta_{j-1}+2 .. beta_j+1 (0 .. for the first strip, .. N_x-1 for the last) with
// no transfer; u~ = u~^(j) on D~^(j), written to Ut.  The solves are independent.
helm_status run_local_solves(helm_dd* h, const double2* F, double2* Ut, int B, const PrecondBufs& bf) {
    const int J = h->J, Nx = (int)h->N[0], Ny = (int)h->N[1];
    const auto& beta = h->beta;
    const bool mixed = h->prec == HELM_PREC_MIXED;
    auto step_of = [&](int j) {
        SweepStep sp{};
        sp.src = F;
        sp.mlo = j > 0 ? beta[j] + 2 : 0;
        sp.mhi = j < J - 1 ? beta[j + 1] + 1 : Nx - 1;
        sp.prev = -1;
        sp.pdir = 0;
        sp.t0 = 0;
        sp.tcoef = 0.0;
        return sp;
    };
    if (h->dim == 3) {
        const int ld = h->slab_ld;
        const size_t vb = (size_t)B * Ny * ld * h->esize;
        char* rbuf = (char*)bf.Y;
        char* ybuf = rbuf + vb;
        for (int j = 0; j < J; ++j) {
            const SweepStep sp = step_of(j);
            SlabWork wk{rbuf, ybuf, nullptr, (const char*)h->d_slab_sxz + h->slab_sxz_off[j] * (int64_t)h->esize,
                        h->ct_sz, h->slab_cy.data(), ld, B, (unsigned*)bf.counters, h->d_status};
            cudaError_t e = mixed ? launch_slab_solve<float2>(h->geom, h->strips[j], nullptr, sp, wk, h->d_pool[0],
                                                              h->stream, &h->timer)
                                  : launch_slab_solve<double2>(h->geom, h->strips[j], nullptr, sp, wk, h->d_pool[0],
                                                               h->stream, &h->timer);
            if (e == cudaSuccess)
                e = mixed ? launch_slab_out<float2>(h->geom, h->strips[j], 1, ybuf, ld, Ut, nullptr, B, h->stream,
                                                    &h->timer)
                          : launch_slab_out<double2>(h->geom, h->strips[j], 1, ybuf, ld, Ut, nullptr, B, h->stream,
                                                     &h->timer);
            if (e != cudaSuccess) return fail_cuda(h, "local strip solves", e);
        }
        return HELM_OK;
    }
    const int ws = work_stride(h);
    const int64_t ystride = (int64_t)B * Ny * ws;
    auto ybuf = [&](int j) { return (char*)bf.Y + j * ystride * (int64_t)h->esize; };
    CK(h, zero_acc2(h, bf.parts, B));
    const int kOutBatch = 8;
    for (int j = 0; j < J; ++j) {
        const SweepStep sp = step_of(j);
        SweepWork wk{ybuf(j), bf.parts, bf.counters, h->d_status, ws, B, h->zrows, nullptr};
        cudaError_t e = mixed ? launch_strip_solve<float2>(h->geom, j, h->strips[j], nullptr, sp, wk, h->d_pool,
                                                           h->stream, &h->timer)
                              : launch_strip_solve<double2>(h->geom, j, h->strips[j], nullptr, sp, wk, h->d_pool,
                                                            h->stream, &h->timer);
        if (e != cudaSuccess) return fail_cuda(h, "local strip solves", e);
        if ((j + 1) % kOutBatch == 0 || j == J - 1) {
            const int n = (j % kOutBatch) + 1;
            OutArgs O{h->geom, 1, j + 1 - n, n, bf.Y, ystride, ws, B, B > 1 ? 4 : 1, Ut, nullptr,
                      j == J - 1 ? 0 : 56};
            CK(h, cudaEventRecord(h->ev_main, h->stream));
            CK(h, cudaStreamWaitEvent(h->side, h->ev_main, 0));
            e = mixed ? launch_outputs<float2>(O, h->d_pool, h->side, &h->timer)
                      : launch_outputs<double2>(O, h->d_pool, h->side, &h->timer);
            if (e != cudaSuccess) return fail_cuda(h, "local strip outputs", e);
        }
    }
    CK(h, cudaEventRecord(h->ev_side, h->side));
    CK(h, cudaStreamWaitEvent(h->stream, h->ev_side, 0));
    return HELM_OK;
}

// Work buffers of the reduced-space routines for B fields: X (a reduced vector extended
// by zero to the grid), Zf (P X), Ut (u~), Rr (the FP64 residual of the outer passes),
// phi and xi (reduced); full fields first, each 256-byte aligned.
struct RedBufs {
    double2 *X, *Zf, *Ut, *Rr, *phi, *xi;
};
helm_status red_reserve(helm_dd* h, int B, RedBufs& rb) {
    const size_t full = (size_t)B * nvol(h) * sizeof(double2), red = (size_t)B * std::max<int64_t>(nred(h), 1) * 16;
    const size_t fa = align256(full), ra = align256(red);
    helm_status s = ws_reserve(h, h->ws_red, 4 * fa + 2 * ra);
    if (s != HELM_OK) return s;
    char* p = (char*)h->ws_red.p;
    rb.X = (double2*)p;
    rb.Zf = (double2*)(p + fa);
    rb.Ut = (double2*)(p + 2 * fa);
    rb.Rr = (double2*)(p + 3 * fa);
    rb.phi = (double2*)(p + 4 * fa);
    rb.xi = (double2*)(p + 4 * fa + ra);
    // X is zero off the interface lines from here on; only its interface columns are written
    CK(h, cudaMemsetAsync(rb.X, 0, full, h->stream));
    return HELM_OK;
}

// Algorithm 2: Ut = u~ and phi = (F - A u~) on the interface lines.
helm_status dev_reduce(helm_dd* h, const double2* F, double2* phi, double2* Ut, int B) {
    size_t sz[kPrecondBufs];
    precond_buf_bytes(h, B, sz);
    helm_status s;
    if ((s = ws_reserve(h, h->ws_Y, sz[2])) != HELM_OK) return s;
    if ((s = ws_reserve(h, h->ws_parts, sz[3])) != HELM_OK) return s;
    PrecondBufs bf{nullptr, nullptr, h->ws_Y.p, h->ws_parts.p, h->d_counters};
    if ((s = run_local_solves(h, F, Ut, B, bf)) != HELM_OK) return s;
    CK(h, launch_stencil_cols(h->geom, Ut, F, nullptr, phi, h->d_icols, (int)h->icols.size(), B, h->stream,
                              &h->timer));
    return HELM_OK;
}

// Algorithm 3 on reduced vectors: out = f - R A P E x (out = R A P E x when f is null),
// with E the extension by zero to the grid and R the restriction to the interface lines.
KrylovOp reduced_op(helm_dd* h, const RedBufs& rb) {
    KrylovOp op;
    op.n = nred(h);
    op.trust_estimate = true;   // dev_solve_reduced forms the true FP64 residual on the whole grid
    const int L = (int)h->icols.size();
    op.residual = [h, rb, L](const double2* x, const double2* f, double2* out, int nb) -> helm_status {
        const int64_t rows = (int64_t)nb * h->N[2] * h->N[1];
        CK(h, launch_scatter_cols(x, rb.X, h->d_icols, L, rows, (int)h->N[0], h->stream, &h->timer));
        helm_status s = dev_precond(h, rb.X, rb.Zf, nb);
        if (s != HELM_OK) return s;
        CK(h, launch_stencil_cols(h->geom, rb.Zf, nullptr, f, out, h->d_icols, L, nb, h->stream, &h->timer));
        return HELM_OK;
    };
    return op;
}

// Full-grid norms of B fields (FP64).
helm_status field_norms(helm_dd* h, const double2* X, int B, int64_t n, std::vector<double>& nrm) {
    helm_status s;
    const int nblk = 304;
    const size_t need = (size_t)B * nblk * sizeof(double2) + (size_t)B * sizeof(double2);
    if ((s = ws_reserve(h, h->ws_small, std::max(need, h->ws_small.bytes))) != HELM_OK) return s;
    double2* partial = (double2*)h->ws_small.p;
    double2* dres = partial + (size_t)B * nblk;
    CK(h, launch_multidot(X, 0, X, 1, B, n, partial, nblk, dres, h->stream, &h->timer));
    std::vector<double2> hr(B);
    CK(h, cudaMemcpyAsync(hr.data(), dres, B * sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    nrm.resize(B);
    for (int b = 0; b < B; ++b) nrm[b] = sqrt(std::max(hr[b].x, 0.0));
    return HELM_OK;
}

// Algorithm 5 in the reduced space for B fields: phi from Algorithm 2, GMRES on
// R A P E xi = phi (Eq. solve_A_reduced, psi = P E xi), u = P E xi + u~ (Algorithm 4).
// Each pass stops GMRES when the reduced residual would bring ||f - A u|| to tol ||f||
// (in mixed precision at 1e-3 of the pass's right-hand side at the tightest); the true
// FP64 residual is then formed on the whole grid and, where it is still above tol ||f||
// (complex64 strip solves leave residuals off the interface lines, which the reduced
// space does not see), the pass is repeated on it (defect correction).
helm_status dev_solve_reduced(helm_dd* h, const double2* F, double2* U, int B, double tol, int m, int maxit,
                              std::vector<int>& iters, std::vector<double>& relres) {
    const int64_t NV = nvol(h);
    RedBufs rb;
    helm_status s;
    if ((s = red_reserve(h, B, rb)) != HELM_OK) return s;
    iters.assign(B, 0);
    relres.assign(B, 0.0);
    std::vector<double> fn, pn, rn;
    if ((s = field_norms(h, F, B, NV, fn)) != HELM_OK) return s;
    for (int b = 0; b < B; ++b)
        if (!std::isfinite(fn[b])) return fail(h, HELM_ENUMERIC, "non-finite right-hand side");
    CK(h, cudaMemsetAsync(U, 0, (size_t)B * NV * sizeof(double2), h->stream));
    const KrylovOp op = reduced_op(h, rb);
    const double2* Rf = F;
    const int kMaxPass = 8;
    bool conv = false;
    for (int pass = 0; pass < kMaxPass && !conv; ++pass) {
        if ((s = dev_reduce(h, Rf, rb.phi, rb.Ut, B)) != HELM_OK) return s;
        if (op.n > 0) {
            if ((s = field_norms(h, rb.phi, B, op.n, pn)) != HELM_OK) return s;
            // complex64 strip solves make the reduced operator linear only up to their
            // rounding, below which GMRES stalls: in mixed precision every pass stops at
            // 1e-3 of its right-hand side and the FP64 passes gain the remaining digits
            const double floor_tol = h->prec == HELM_PREC_MIXED ? 1e-3 : 1e-14;
            std::vector<double> tv(B);
            for (int b = 0; b < B; ++b) {
                const double target = (pass == 0 ? 1.0 : 0.5) * tol * fn[b];
                tv[b] = pn[b] > 0 ? std::min(0.5, std::max(target / pn[b], floor_tol)) : 1.0;
            }
            std::vector<int> it;
            std::vector<double> rr;
            const int left = std::max(1, maxit - *std::max_element(iters.begin(), iters.end()));
            s = dev_gmres(h, op, rb.phi, rb.xi, B, tol, m, left, it, rr, &tv);
            if (s != HELM_OK && s != HELM_ENOTCONV) return s;
            for (int b = 0; b < B; ++b) iters[b] += it[b];
            // Algorithm 4: u += P E xi + u~
            CK(h, launch_scatter_cols(rb.xi, rb.X, h->d_icols, (int)h->icols.size(), (int64_t)B * h->N[2] * h->N[1],
                                      (int)h->N[0], h->stream, &h->timer));
            if ((s = dev_precond(h, rb.X, rb.Zf, B)) != HELM_OK) return s;
            CK(h, launch_add(U, rb.Zf, (int64_t)B * NV, h->stream, &h->timer));
        }
        CK(h, launch_add(U, rb.Ut, (int64_t)B * NV, h->stream, &h->timer));
        // the true residual f - A u on the whole grid (FP64)
        if ((s = dev_stencil(h, U, F, rb.Rr, B)) != HELM_OK) return s;
        if ((s = field_norms(h, rb.Rr, B, NV, rn)) != HELM_OK) return s;
        conv = true;
        for (int b = 0; b < B; ++b) {
            if (!std::isfinite(rn[b])) return fail(h, HELM_ENUMERIC, "non-finite residual norm");
            relres[b] = fn[b] > 0 ? rn[b] / fn[b] : 0.0;
            if (!(relres[b] <= tol)) conv = false;
        }
        if (*std::max_element(iters.begin(), iters.end()) >= maxit) break;
        Rf = rb.Rr;
    }
    return conv ? HELM_OK : fail(h, HELM_ENOTCONV, "reduced-space GMRES did not reach the tolerance");
}

// Device view of a caller's input array (host arrays are copied into ws).
helm_status stage_in(helm_dd* h, const double* p, size_t bytes, helm_dd::Ws& ws, const double2** out) {
    if (is_device_ptr(p)) {
        if (misaligned16(p)) return fail(h, HELM_EINVAL, "device fields must be 16-byte aligned (complex128)");
        *out = (const double2*)p;
        return HELM_OK;
    }
    helm_status s = ws_reserve(h, ws, bytes);
    if (s != HELM_OK) return s;
    CK(h, cudaMemcpyAsync(ws.p, p, bytes, cudaMemcpyHostToDevice, h->stream));
    *out = (const double2*)ws.p;
    return HELM_OK;
}
// Device buffer for a caller's output array: the array itself when it is on the device,
// else ws (copied back by unstage_out).
helm_status stage_out(helm_dd* h, double* p, size_t bytes, helm_dd::Ws& ws, double2** out) {
    if (is_device_ptr(p)) {
        if (misaligned16(p)) return fail(h, HELM_EINVAL, "device fields must be 16-byte aligned (complex128)");
        *out = (double2*)p;
        return HELM_OK;
    }
    helm_status s = ws_reserve(h, ws, bytes);
    if (s != HELM_OK) return s;
    *out = (double2*)ws.p;
    return HELM_OK;
}
helm_status unstage_out(helm_dd* h, double* p, const double2* dev, size_t bytes) {
    if ((const void*)p != (const void*)dev)
        CK(h, cudaMemcpyAsync(p, dev, bytes, cudaMemcpyDeviceToHost, h->stream));
    return HELM_OK;
}

// Right-hand sides per panel of the reduced solve (at most the handle's setting): per
// right-hand side four full fields
// of its own, the preconditioner's two, the strip chain solutions, and m+4 reduced vectors.
int panel_width_reduced(helm_dd* h, int nrhs, int m) {
    if (h->panel > 0) nrhs = std::min(h->panel, nrhs);   // the caller's cap
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { cudaGetLastError(); return nrhs; }
    for (auto* w : {&h->ws_V, &h->ws_G, &h->ws_Y, &h->ws_parts, &h->ws_kry, &h->ws_small, &h->ws_red}) fr += w->bytes;
    size_t sz[kPrecondBufs];
    precond_buf_bytes(h, 1, sz);
    const size_t field = (size_t)nvol(h) * sizeof(double2);
    const size_t per = 4 * field + sz[0] + sz[1] + sz[2] + sz[3] + (size_t)(m + 4) * nred(h) * 16 + 4096;
    const size_t fit = (size_t)(0.85 * (double)fr) / per;
    const int Bp = (int)std::max<size_t>(1, std::min<size_t>((size_t)nrhs, fit));
    release_if_short(h, (size_t)Bp * per);
    return Bp;
}

}  // namespace

extern "C" {

helm_status helm_dd_solve(helm_dd* h, const double* rhs, double* u, int nrhs, double tol, int restart, int maxit,
                          helm_rhs_info* info) {
    if (!h || !rhs || !u || nrhs < 1 || !(tol > 0) || restart < 1 || maxit < 1) return HELM_EINVAL;
    if (!h->factored) return fail(h, HELM_ESTATE, "solve before factor");
    const auto t0 = std::chrono::steady_clock::now();
    const size_t bytes = (size_t)nrhs * nvol(h) * sizeof(double2);
    const bool din = is_device_ptr(rhs), dout = is_device_ptr(u);
    if ((din && misaligned16(rhs)) || (dout && misaligned16(u)))
        return fail(h, HELM_EINVAL, "device fields must be 16-byte aligned (complex128)");
    helm_status s;
    const double2* F = (const double2*)rhs;
    double2* U = (double2*)u;
    if (!din) {
        if ((s = ws_reserve(h, h->ws_io_in, bytes)) != HELM_OK) return s;
        CK(h, cudaMemcpyAsync(h->ws_io_in.p, rhs, bytes, cudaMemcpyHostToDevice, h->stream));
        F = (const double2*)h->ws_io_in.p;
    }
    if (!dout) {
        if ((s = ws_reserve(h, h->ws_io_out, bytes)) != HELM_OK) return s;
        U = (double2*)h->ws_io_out.p;
    }
    std::vector<int> iters(nrhs), it_p;
    std::vector<double> relres(nrhs), rr_p;
    helm_status st = HELM_OK;
    const int Bp = panel_width(h, nrhs, restart, din ? 0 : 2);
    const int64_t NV = nvol(h);
    for (int b0 = 0; b0 < nrhs; b0 += Bp) {   // right-hand sides in panels of Bp
        const int nb = std::min(Bp, nrhs - b0);
        helm_status sp = dev_fgmres(h, F + (int64_t)b0 * NV, U + (int64_t)b0 * NV, nb, tol, restart, maxit, it_p, rr_p);
        if (sp != HELM_OK && sp != HELM_ENOTCONV) return sp;
        if (sp == HELM_ENOTCONV) st = sp;
        for (int b = 0; b < nb; ++b) { iters[b0 + b] = it_p[b]; relres[b0 + b] = rr_p[b]; }
    }
    helm_status ds = check_device_status(h);
    if (ds != HELM_OK) return ds;
    if (!dout) CK(h, cudaMemcpyAsync(u, U, bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info)
        for (int b = 0; b < nrhs; ++b) info[b] = helm_rhs_info{iters[b], relres[b], ms};
    return st;
}

int helm_dd_interface_lines(const helm_dd* h, int* cols, int cap) {
    if (!h) return 0;
    for (int i = 0; i < (int)h->icols.size() && i < cap && cols; ++i) cols[i] = h->icols[i];
    return (int)h->icols.size();
}

helm_status helm_dd_reduce_rhs(helm_dd* h, const double* f, double* phi, double* ut, int nrhs) {
    if (!h || !f || nrhs < 1) return HELM_EINVAL;
    if (!h->factored) return fail(h, HELM_ESTATE, "reduce_rhs before factor");
    const int64_t NR = nred(h);
    if (NR > 0 && !phi) return HELM_EINVAL;
    const size_t fb = (size_t)nrhs * nvol(h) * sizeof(double2), rbytes = (size_t)nrhs * NR * sizeof(double2);
    helm_status s;
    const double2* F;
    double2* Phi = nullptr;
    if ((s = stage_in(h, f, fb, h->ws_io_in, &F)) != HELM_OK) return s;
    if (NR > 0 && (s = stage_out(h, phi, rbytes, h->ws_io_out, &Phi)) != HELM_OK) return s;
    RedBufs rb;
    if ((s = red_reserve(h, nrhs, rb)) != HELM_OK) return s;
    if ((s = dev_reduce(h, F, Phi, rb.Ut, nrhs)) != HELM_OK) return s;
    if ((s = check_device_status(h)) != HELM_OK) return s;
    if (NR > 0 && (s = unstage_out(h, phi, Phi, rbytes)) != HELM_OK) return s;
    if (ut) CK(h, cudaMemcpyAsync(ut, rb.Ut, fb, is_device_ptr(ut) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return HELM_OK;
}

helm_status helm_dd_apply_AP_reduced(helm_dd* h, const double* in, double* out, int nrhs) {
    if (!h || !in || !out || nrhs < 1) return HELM_EINVAL;
    if (!h->factored) return fail(h, HELM_ESTATE, "apply_AP_reduced before factor");
    const int64_t NR = nred(h);
    if (NR == 0) return HELM_OK;
    const size_t rbytes = (size_t)nrhs * NR * sizeof(double2);
    helm_status s;
    const double2* X;
    double2* Y;
    if ((s = stage_in(h, in, rbytes, h->ws_io_in, &X)) != HELM_OK) return s;
    if ((s = stage_out(h, out, rbytes, h->ws_io_out, &Y)) != HELM_OK) return s;
    if ((const void*)X == (const void*)Y) return fail(h, HELM_EINVAL, "apply_AP_reduced needs distinct buffers");
    RedBufs rb;
    if ((s = red_reserve(h, nrhs, rb)) != HELM_OK) return s;
    const KrylovOp op = reduced_op(h, rb);
    if ((s = op.residual(X, nullptr, Y, nrhs)) != HELM_OK) return s;
    if ((s = check_device_status(h)) != HELM_OK) return s;
    if ((s = unstage_out(h, out, Y, rbytes)) != HELM_OK) return s;
    CK(h, cudaStreamSynchronize(h->stream));
    return HELM_OK;
}

helm_status helm_dd_solve_reduced(helm_dd* h, const double* rhs, double* u, int nrhs, double tol, int restart,
                                  int maxit, helm_rhs_info* info) {
    if (!h || !rhs || !u || nrhs < 1 || !(tol > 0) || restart < 1 || maxit < 1) return HELM_EINVAL;
    if (!h->factored) return fail(h, HELM_ESTATE, "solve_reduced before factor");
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t NV = nvol(h);
    const size_t bytes = (size_t)nrhs * NV * sizeof(double2);
    helm_status s;
    const double2* F;
    double2* U;
    if ((s = stage_in(h, rhs, bytes, h->ws_io_in, &F)) != HELM_OK) return s;
    if ((s = stage_out(h, u, bytes, h->ws_io_out, &U)) != HELM_OK) return s;
    std::vector<int> iters(nrhs), it_p;
    std::vector<double> relres(nrhs), rr_p;
    helm_status st = HELM_OK;
    const int Bp = panel_width_reduced(h, nrhs, restart);
    for (int b0 = 0; b0 < nrhs; b0 += Bp) {   // right-hand sides in panels of Bp
        const int nb = std::min(Bp, nrhs - b0);
        helm_status sp = dev_solve_reduced(h, F + (int64_t)b0 * NV, U + (int64_t)b0 * NV, nb, tol, restart, maxit,
                                           it_p, rr_p);
        if (sp != HELM_OK && sp != HELM_ENOTCONV) return sp;
        if (sp == HELM_ENOTCONV) st = sp;
        for (int b = 0; b < nb; ++b) { iters[b0 + b] = it_p[b]; relres[b0 + b] = rr_p[b]; }
    }
    helm_status ds = check_device_status(h);
    if (ds != HELM_OK) return ds;
    if ((s = unstage_out(h, u, U, bytes)) != HELM_OK) return s;
    CK(h, cudaStreamSynchronize(h->stream));
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info)
        for (int b = 0; b < nrhs; ++b) info[b] = helm_rhs_info{iters[b], relres[b], ms};
    return st;
}

helm_status helm_dd_gradient(helm_dd* h, const int64_t* src_idx, int nsrc, const int64_t* rec_idx, int nrec,
                             const double* d, double tol, double* misfit, double* grad_m) {
    if (!h || !src_idx || !rec_idx || !d || !misfit || nsrc < 1 || nrec < 1) return HELM_EINVAL;
    if (!h->factored) return fail(h, HELM_ESTATE, "gradient before factor");
    const int64_t NV = nvol(h);
    for (int i = 0; i < nsrc; ++i)
        if (src_idx[i] < 0 || src_idx[i] >= NV) return fail(h, HELM_EINVAL, "source index out of range");
    for (int i = 0; i < nrec; ++i)
        if (rec_idx[i] < 0 || rec_idx[i] >= NV) return fail(h, HELM_EINVAL, "receiver index out of range");
    const bool want_grad = grad_m != nullptr;
    const int Bp = panel_width(h, nsrc, 20, want_grad ? 3 : 2);
    const size_t vb = (size_t)Bp * NV * sizeof(double2);
    helm_status s;
    // ws_grad holds F/Q, U, MU (one panel each), gpad, gint, the receiver and scatter
    // index / value arrays and the gathered values, each on a 256-byte boundary (the
    // complex128 arrays need 16-byte alignment whatever the counts)
    const int64_t nint = h->n[0] * h->n[1] * h->n[2];
    const size_t part[9] = {vb, vb, want_grad ? vb : 0, (size_t)NV * sizeof(double), (size_t)nint * sizeof(double),
                            (size_t)nrec * sizeof(int64_t), (size_t)Bp * nrec * sizeof(int64_t),
                            (size_t)Bp * nrec * sizeof(double2), (size_t)Bp * nrec * sizeof(double2)};
    size_t off[10];
    off[0] = 0;
    for (int i = 0; i < 9; ++i) off[i + 1] = off[i] + ((part[i] + 255) & ~(size_t)255);
    if ((s = ws_reserve(h, h->ws_grad, off[9])) != HELM_OK) return s;
    char* wb = (char*)h->ws_grad.p;
    double2* FQ = (double2*)(wb + off[0]);
    double2* U = (double2*)(wb + off[1]);
    double2* MU = (double2*)(wb + off[2]);
    double* gpad = (double*)(wb + off[3]);
    double* gint = (double*)(wb + off[4]);
    int64_t* drec = (int64_t*)(wb + off[5]);
    int64_t* dsi = (int64_t*)(wb + off[6]);
    double2* dsv = (double2*)(wb + off[7]);
    double2* gath = (double2*)(wb + off[8]);
    std::vector<double2> dd((size_t)nsrc * nrec);
    if (is_device_ptr(d)) CK(h, cudaMemcpy(dd.data(), d, dd.size() * sizeof(double2), cudaMemcpyDeviceToHost));
    else memcpy(dd.data(), d, dd.size() * sizeof(double2));
    CK(h, cudaMemcpyAsync(drec, rec_idx, nrec * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
    if (want_grad) CK(h, cudaMemsetAsync(gpad, 0, (size_t)NV * sizeof(double), h->stream));
    const double amp = 1.0 / pow(h->h, h->dim);   // sources: discrete deltas 1/h^dim
    const int Nx = (int)h->N[0], Ny = (int)h->N[1];
    std::vector<int64_t> si((size_t)Bp * nrec);
    std::vector<double2> sv((size_t)Bp * nrec), ur((size_t)Bp * nrec);
    std::vector<int> iters;
    std::vector<double> relres;
    double J = 0.0;
    // Sources in panels of Bp (as many as the free device memory holds): the forward
    // fields of one panel exist only until that panel's adjoint solves are done.
    for (int s0 = 0; s0 < nsrc; s0 += Bp) {
        const int nb = std::min(Bp, nsrc - s0);
        CK(h, cudaMemsetAsync(FQ, 0, (size_t)nb * NV * sizeof(double2), h->stream));
        for (int b = 0; b < nb; ++b) { si[b] = src_idx[s0 + b]; sv[b] = make_double2(amp, 0.0); }
        CK(h, cudaMemcpyAsync(dsi, si.data(), nb * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaMemcpyAsync(dsv, sv.data(), nb * sizeof(double2), cudaMemcpyHostToDevice, h->stream));
        CK(h, launch_scatter(FQ, NV, dsi, dsv, 1, nb, h->stream));
        helm_status st = dev_fgmres(h, FQ, U, nb, tol, 20, 400, iters, relres);
        if (st != HELM_OK) return st;
        // residual at the receivers and the misfit
        CK(h, launch_gather(U, NV, drec, nrec, nb, gath, h->stream));
        CK(h, cudaMemcpyAsync(ur.data(), gath, (size_t)nb * nrec * sizeof(double2), cudaMemcpyDeviceToHost,
                              h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        // adjoint right-hand sides q = S^-1 conj(R^T r): repeated receivers of a source
        // are summed here, so the scatter writes each point once
        for (int b = 0; b < nb; ++b) {
            std::vector<std::pair<int64_t, cd>> acc;
            for (int r = 0; r < nrec; ++r) {
                const double2 u0 = ur[(size_t)b * nrec + r], d0 = dd[(size_t)(s0 + b) * nrec + r];
                const cd res(u0.x - d0.x, u0.y - d0.y);
                J += 0.5 * std::norm(res);
                bool found = false;
                for (auto& pr : acc)
                    if (pr.first == rec_idx[r]) { pr.second += res; found = true; }
                if (!found) acc.push_back({rec_idx[r], res});
            }
            for (int r = 0; r < nrec; ++r) {
                const auto& pr = acc[std::min(r, (int)acc.size() - 1)];   // unused slots repeat the last point
                const int64_t p = pr.first;
                const int x = (int)(p % Nx), y = (int)((p / Nx) % Ny), z = (int)(p / ((int64_t)Nx * Ny));
                cd S = (1.0 / h->gx_int[x]) * (1.0 / h->gy_int[y]);
                if (h->dim == 3) S *= 1.0 / h->gz_int[z];
                const cd q = std::conj(pr.second) / S;
                si[(size_t)b * nrec + r] = p;
                sv[(size_t)b * nrec + r] = make_double2(q.real(), q.imag());
            }
        }
        if (!want_grad) continue;
        CK(h, cudaMemsetAsync(FQ, 0, (size_t)nb * NV * sizeof(double2), h->stream));
        CK(h, cudaMemcpyAsync(dsi, si.data(), (size_t)nb * nrec * sizeof(int64_t), cudaMemcpyHostToDevice,
                              h->stream));
        CK(h, cudaMemcpyAsync(dsv, sv.data(), (size_t)nb * nrec * sizeof(double2), cudaMemcpyHostToDevice,
                              h->stream));
        CK(h, launch_scatter(FQ, NV, dsi, dsv, nrec, nb, h->stream));
        st = dev_fgmres(h, FQ, MU, nb, tol, 20, 400, iters, relres);
        if (st != HELM_OK) return st;
        CK(h, launch_grad_accum(U, MU, h->geom, nb, gpad, h->stream));
    }
    if (want_grad) {
        CK(h, launch_fold(gpad, gint, h->dim, (int)h->n[0], (int)h->n[1], (int)h->n[2], h->w_outer, h->stream));
        if (is_device_ptr(grad_m))
            CK(h, cudaMemcpyAsync(grad_m, gint, nint * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        else
            CK(h, cudaMemcpyAsync(grad_m, gint, nint * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    *misfit = J;
    return HELM_OK;
}

double helm_dd_precond_factor_bytes(const helm_dd* h) {
    if (!h) return 0.0;
    double b = 0.0;
    for (int j = 0; j < h->J; ++j) {
        const double n = (double)h->strips[j].W * h->N[2];   // unknowns of a block (N_z = 1 in 2-D)
        const double blk = (double)h->N[1] * n * n * h->esize;
        b += 2.0 * blk * (j < h->J - 1 ? 2.0 : 1.0);
    }
    return b;
}

void helm_dd_dims(const helm_dd* h, int64_t N[3]) {
    if (!h || !N) return;
    for (int a = 0; a < 3; ++a) N[a] = h->N[a];
}

int helm_dd_strip_widths(const helm_dd* h, int* W, int cap) {
    if (!h) return 0;
    for (int j = 0; j < h->J && j < cap && W; ++j) W[j] = h->strips[j].W;
    return h->J;
}

int helm_dd_interfaces(const helm_dd* h, int* beta, int cap) {
    if (!h) return 0;
    for (int j = 0; j <= h->J && j < cap && beta; ++j) beta[j] = h->beta[j];
    return h->J + 1;
}

void helm_dd_destroy(helm_dd* h) {
    if (!h) return;
    if (!h->dev_ready && !h->own_stream) { delete h; return; }
    if (h->stream) cudaStreamSynchronize(h->stream);
    h->timer.flush();
    cudaFree(h->d_c);
    cudaFree(h->d_k2);
    cudaFree(h->d_tab);
    cudaFree(h->d_strips);
    cudaFree(h->d_ints);
    cudaFree(h->d_status);
    for (auto p : h->d_pool) cudaFree(p);
    cudaFree(h->d_ct);
    cudaFree(h->d_slab_sxz);
    cudaFree(h->d_counters);
    cudaFree(h->d_icols);
    cudaFree(h->d_rab);
    for (auto* w : {&h->ws_V, &h->ws_G, &h->ws_Y, &h->ws_parts, &h->ws_io_in, &h->ws_io_out, &h->ws_io_aux,
                    &h->ws_kry, &h->ws_small, &h->ws_grad, &h->ws_red})
        ws_free(*w);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->ev_main) cudaEventDestroy(h->ev_main);
    if (h->ev_side) cudaEventDestroy(h->ev_side);
    for (auto cs : h->cstream) if (cs) cudaStreamDestroy(cs);
    for (auto ev : h->cev) if (ev) cudaEventDestroy(ev);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    cudaGetLastError();
    delete h;
}

const char* helm_dd_last_error(const helm_dd* h) { return h ? h->err.c_str() : "null handle"; }

extern "C" helm_status helm_dd_apply_precond_noalloc(helm_dd* h, const double* in, double* out, int nrhs) {
    if (!h || !in || !out || nrhs < 1) return HELM_EINVAL;
    if (!h->factored) return fail(h, HELM_ESTATE, "apply_precond_noalloc before factor");
    if (!is_device_ptr(in) || !is_device_ptr(out))
        return fail(h, HELM_EINVAL, "apply_precond_noalloc takes device pointers only (host staging would allocate)");
    if (misaligned16(in) || misaligned16(out))
        return fail(h, HELM_EINVAL, "device fields must be 16-byte aligned (complex128)");
    if ((const void*)in == (const void*)out)
        return fail(h, HELM_EINVAL, "apply_precond_noalloc needs distinct input and output buffers");
    size_t sz[kPrecondBufs];
    precond_buf_bytes(h, nrhs, sz);
    size_t off[kPrecondBufs + 1];
    size_t total = 0;
    for (int i = 0; i < kPrecondBufs; ++i) { off[i] = total; total += align256(sz[i]); }
    off[kPrecondBufs] = total;
    total += align256(h->counter_bytes);
    if (total > kNoAllocScratchBytes)
        return fail(h, HELM_EINVAL, "apply_precond_noalloc needs " + std::to_string(total) +
                                        " bytes of scratch; the static limit is " +
                                        std::to_string(kNoAllocScratchBytes) + " (use fewer right-hand sides)");
    if (!h->noalloc_base) return fail(h, HELM_ESTATE, "no-allocation scratch not set up on this device");
    unsigned char* b = (unsigned char*)h->noalloc_base;
    PrecondBufs bf{(double2*)(b + off[0]), (double2*)(b + off[1]), b + off[2], b + off[3],
                   (int*)(b + off[kPrecondBufs])};
    // the array keeps whatever the previous call left: the arrival counters must start at zero
    CK(h, cudaMemsetAsync(bf.counters, 0, h->counter_bytes, h->stream));
    helm_status s = run_precond(h, (const double2*)in, (double2*)out, nrhs, bf);
    if (s != HELM_OK) return s;
    return check_device_status(h);
}

}  // extern "C"
