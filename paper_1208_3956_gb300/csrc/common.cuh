// Shared device-side definitions of the helm_dd library: complex arithmetic on
// float2 / double2, strip descriptors and kernel argument blocks.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace helm {

// ---------------------------------------------------------------- complex ops
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc + a*b with fused multiply-adds
__host__ __device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
    acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}
__host__ __device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
__host__ __device__ __forceinline__ float2 cneg(float2 a) { return make_float2(-a.x, -a.y); }
__host__ __device__ __forceinline__ double2 cneg(double2 a) { return make_double2(-a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
// a += v by two atomic adds (concurrent adds are summed in arrival order)
__device__ __forceinline__ void catomic_add(float2* a, float2 v) {
    atomicAdd(&a->x, v.x);
    atomicAdd(&a->y, v.y);
}
__device__ __forceinline__ void catomic_add(double2* a, double2 v) {
    atomicAdd(&a->x, v.x);
    atomicAdd(&a->y, v.y);
}
__host__ __device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// 1 / a, scaled to avoid overflow of |a|^2
__host__ __device__ __forceinline__ float2 cinv(float2 a) {
    float s = fmaxf(fabsf(a.x), fabsf(a.y));
    float ar = a.x / s, ai = a.y / s;
    float d = s * (ar * ar + ai * ai);
    return make_float2(ar / d, -ai / d);
}
__host__ __device__ __forceinline__ double2 cinv(double2 a) {
    double s = fmax(fabs(a.x), fabs(a.y));
    double ar = a.x / s, ai = a.y / s;
    double d = s * (ar * ar + ai * ai);
    return make_double2(ar / d, -ai / d);
}

template <typename C> struct CT;
template <> struct CT<float2> {
    using R = float;
    __host__ __device__ static float2 zero() { return make_float2(0.f, 0.f); }
    __host__ __device__ static float2 from(double2 a) { return make_float2((float)a.x, (float)a.y); }
};
template <> struct CT<double2> {
    using R = double;
    __host__ __device__ static double2 zero() { return make_double2(0.0, 0.0); }
    __host__ __device__ static double2 from(double2 a) { return a; }
};
__host__ __device__ __forceinline__ double2 to_d2(float2 a) { return make_double2(a.x, a.y); }
__host__ __device__ __forceinline__ double2 to_d2(double2 a) { return a; }

// ------------------------------------------------------------ problem layout
// One strip of the decomposition along x (0-based j = 0..J-1).  Its grid is
// lpml added PML columns, the physical padded columns lo..hi (hi is the overlap
// column beta_{j+1}+1 for j < J-1), then rpml added columns.  Strip-local column
// c corresponds to padded column lo - lpml + c.
struct StripDev {
    int W, lo, hi, lpml, rpml, j;
    int64_t tab;   // offset of this strip's x tables: alpha at integer points (W), then half points (W+1)
    int64_t fac;   // element offset of this strip's blocks in the factor pools (Ny blocks of BS)
    int64_t red;   // element offset of this strip's reduced-system blocks ((P-1) blocks of BS)
    int64_t xf;    // element offset of this strip's transfer composites (Ny rows of 16 spld(W))
    int64_t bs;    // elements per stored W x W block (column-major, padded to 16 bytes)
    int64_t ctab;  // offset of this strip's s_x(c) (W entries) in the working-precision table
    int nj;        // columns per lane in the sweep products (W <= 4 nj)
    int ld;        // leading dimension of the sweep-layout blocks (4 nj + 2)
    int olo[2], ohi[2];   // padded output columns of the forward (0) and backward (1) sweeps
    int xc[4];            // strip-local transfer columns: forward to0, to1, backward to0, to1
};

// Sweep layout of the W x W blocks Sinv, Rinv, E, F: row-major with leading
// dimension ld (>= 4 nj >= W), columns W..ld-1 zero.  Element (r, a) sits at
// r * ld + a, so a lane owning row r and columns g*nj .. g*nj+nj-1 reads one
// contiguous run; the +2 padding spreads the rows of a warp over the banks.
__host__ __device__ __forceinline__ int sweep_nj(int W) {
    return W <= 32 ? 8 : W <= 40 ? 10 : W <= 48 ? 12 : W <= 56 ? 14 : 16;
}

// Spikes GT / GB (and GT2 / GB2) are stored row-major, W rows of spld(W)
// entries: an even row length keeps every row 16-byte aligned for bulk copies.
__host__ __device__ __forceinline__ int spld(int W) { return (W + 1) & ~1; }

// Global geometry and tables (device pointers, FP64).
struct Geom {
    int dim;
    int Nx, Ny, Nz;
    int J, P;                  // strips, chunks along y
    double h, inv_h2, omega;
    const double* k2;          // [Nz][Ny][Nx]
    const double2* gx_int;     // alpha at integer points, x / y / z
    const double2* gx_half;    // alpha at half points m-1/2, m = 0..N
    const double2* gy_int;
    const double2* gy_half;
    const double2* gz_int;
    const double2* gz_half;
    const double2* stab;       // per-strip x tables (see StripDev::tab)
    const StripDev* strips;
    const int* r0;             // chunk p covers rows r0[p] .. r1[p]-1; separator p is row r1[p]
    const int* r1;
    const int* rowmap;         // row k -> chunk p (>= 0) or separator q as -(q+1)
    // working-precision (complex64 or complex128) tables for the sweep:
    //   ct[ct_sy + k] = s_y(k) = 1/alpha_y(y_k)          (k < Ny)
    //   ct[ct_cy + k] = -alpha_y(y_{k-1/2}) / h^2       (k <= Ny)
    //   ct[strip.ctab + c] = s_x(c) on the strip grid
    // so that the y-coupling of rows k-1, k is C_k(c) = s_x(c) ct[ct_cy + k]
    // and the right-hand-side scaling is s_x(c) s_y(k).
    const void* ct;
    int64_t ct_sy, ct_cy;
    int64_t ct_sz;             // 3-D strips: ct[ct_sz + z] = s_z(z)
    // second level of nested dissection on the separator system: groups
    // g = 0..G-1 of separators gq0[g] .. gq1[g]-1; level-2 separator r (r < G-1)
    // is separator gq1[r]; sepmap[q] = group of separator q, or -(r+1) for a
    // level-2 separator.  G = 1: one group, no level 2.
    int G;
    const int* gq0;
    const int* gq1;
    const int* sepmap;
    // per chunk p, two int4: {r0, r1, gA, gB}, {raA, rbA, raB, rbB}: gA / gB is the
    // group of the separator above / below the chunk (-1: none, level 2, or G = 1),
    // ra / rb the rows of the level-2 separators above and below that group
    const int4* cmeta;
    // entries of the paper-form stencil per axis (Section 2.2), three per grid index i:
    //   {-a(i) a(i-1/2) / h^2, a(i) (a(i-1/2) + a(i+1/2)) / h^2, -a(i) a(i+1/2) / h^2}
    // and, per axis, the index range [f0, f1) where they are exactly {-1, 2, -1} / h^2
    // (outside every PML)
    const double2* stc_x;
    const double2* stc_y;
    const double2* stc_z;
    int fx0, fx1, fy0, fy1, fz0, fz1;
    // Robin transmission (Section 4.4; null with PML transmission): rab[j * Ny + k] = a/b
    // of the discrete Robin condition on row k next to padded column beta_j + 1, the
    // boundary column shared by strip j (its first) and strip j-1 (its last), j = 1..J-1;
    // a = 1/h + ik/2, b = -1/h + ik/2
    const double2* rab;
};

__host__ __device__ __forceinline__ int imin(int a, int b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int imax(int a, int b) { return a > b ? a : b; }

}  // namespace helm
