// Internal declarations shared by the kernels and the C-ABI host code of liblbm.so.
//
// Data layout in HBM (pull scheme, two buffers A/B swapped every step). Each buffer holds the
// post-collision populations of one step at the cell that computed them; the next step pulls
// direction d from cell x - v_d.
//   MM: 12 direction groups; group d = p*4 + (i-1) is one float4 per cell:
//       (f^(0)_{d,j=0}, f^(0)_{d,j=1}, f^(1)_{d,j=0}, f^(1)_{d,j=1}), array [12][n].
//       Optional rest population f_0^(0) as float[n] (double-buffered) and f_0^(1) as float[n].
//   HV: 6 directions; direction i is a float4 (e_x, e_y, e_z, h_x) in array [6][n] and a float2
//       (h_y, h_z) in a second array [6][n].
// All 16-byte groups are 16-byte aligned whatever the neighbour shift, so every pull is one
// vector load per group.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace lbm {

constexpr int kMaxSources = 16;
constexpr int kBlock = 256;

enum MediaMode { kUniform = 0, kTable = 1, kPerCell = 2 };

struct Geometry {
    int nx, ny, nz;
    int n;  // nx * ny * nz, < 2^31
};

// Media as the kernels see it; (eps_r, mu_r, sigma) per cell.
struct MediaView {
    float4 uniform;          // kUniform: (eps_r, mu_r, sigma, 0)
    const uint8_t* id;       // kTable: material id per cell
    const float4* table;     // kTable: (eps_r, mu_r, sigma, 0) per material
    const float* eps_r;      // kPerCell
    const float* mu_r;
    const float* sigma;
};

// Merged list of cells touched by sources ("special cells"), sorted by cell index.
struct SourceView {
    int n_special;
    const int* cell;            // [n_special]
    const int* entry_begin;     // [n_special + 1] CSR offsets into the current entries
    const int* entry_src;       // source slot of each current entry
    const float* entry_w;       // 3 weights per current entry
    const uint32_t* impose_mask;  // bit k set: source slot k imposes fields at this cell
};

// Per-step source values s_k(t) and the constant imposed-field vectors of each slot.
struct SourceScalars {
    float s[kMaxSources];
    float E0[kMaxSources][3];
    float B0[kMaxSources][3];
};

struct StepArgs {
    const void* fin;    // MM: float4[12][n]; HV: float4[6][n]
    void* fout;
    const void* fin2;   // HV: float2[6][n]
    void* fout2;
    const float* rho_in;  // MM rest population f_0^(0) (track_rho), else null
    float* rho_out;
    Geometry g;
    int media_mode;
    MediaView media;
    SourceView sv;
    SourceScalars sc;
    float eps0, mu0;
};

// Field output: for each selected field a 3 x n block; null pointers are skipped.
struct FieldsOut {
    float* E;
    float* B;
    float* D;
    float* H;
    float* J;
};

// --- compile-time loop ---------------------------------------------------------------------
template <int I, int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

// Signed term c * x for a compile-time c in {-1, 0, 1}; adds nothing for c = 0.
template <int C>
__device__ __forceinline__ void acc(float& sum, float x) {
    if constexpr (C > 0) sum += x;
    else if constexpr (C < 0) sum -= x;
}

// Pairwise (tree) sum of t[B..E) with compile-time bounds. The moment sums use it: on long runs
// it halves the accumulated FP32 error of a left-to-right sum at no extra cost.
template <int B, int E, int N>
__device__ __forceinline__ float pairwise_sum(const float (&t)[N]) {
    static_assert(E > B, "empty sum");
    if constexpr (E - B == 1) {
        return t[B];
    } else {
        constexpr int M = B + (E - B) / 2;
        return pairwise_sum<B, M>(t) + pairwise_sum<M, E>(t);
    }
}

// --- periodic neighbour addressing ---------------------------------------------------------
// Linear-index contributions of the three coordinates shifted by -1, 0, +1 with periodic wrap.
struct Neighbourhood {
    int xo[3], yo[3], zo[3];
};

__device__ __forceinline__ Neighbourhood neighbourhood(const Geometry& g, int i) {
    const int nxy = g.nx * g.ny;
    const int z = i / nxy;
    const int r = i - z * nxy;
    const int y = r / g.nx;
    const int x = r - y * g.nx;
    Neighbourhood h;
    h.xo[0] = x == 0 ? g.nx - 1 : x - 1;
    h.xo[1] = x;
    h.xo[2] = x == g.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
    h.yo[0] = ym * g.nx;
    h.yo[1] = y * g.nx;
    h.yo[2] = yp * g.nx;
    const int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
    h.zo[0] = zm * nxy;
    h.zo[1] = z * nxy;
    h.zo[2] = zp * nxy;
    return h;
}

// Index of the cell at offset (sx, sy, sz) in {-1, 0, 1}^3.
template <int SX, int SY, int SZ>
__device__ __forceinline__ int shifted(const Neighbourhood& h) {
    return h.xo[SX + 1] + h.yo[SY + 1] + h.zo[SZ + 1];
}

template <int M>
__device__ __forceinline__ float3 load_material(const MediaView& m, int i) {
    if constexpr (M == kUniform) {
        return make_float3(m.uniform.x, m.uniform.y, m.uniform.z);
    } else if constexpr (M == kTable) {
        const float4 t = __ldg(&m.table[__ldg(&m.id[i])]);
        return make_float3(t.x, t.y, t.z);
    } else {
        return make_float3(__ldg(&m.eps_r[i]), __ldg(&m.mu_r[i]), __ldg(&m.sigma[i]));
    }
}

// External current and imposed fields of special cell m at the current step.
struct CellSource {
    float3 J;
    float3 E;
    float3 B;
    bool imposed;
};

__device__ __forceinline__ CellSource cell_source(const SourceView& sv, const SourceScalars& sc, int m) {
    CellSource cs;
    cs.J = make_float3(0.f, 0.f, 0.f);
    cs.E = make_float3(0.f, 0.f, 0.f);
    cs.B = make_float3(0.f, 0.f, 0.f);
    const int b = sv.entry_begin[m], e = sv.entry_begin[m + 1];
    for (int k = b; k < e; ++k) {
        const float s = sc.s[sv.entry_src[k]];
        cs.J.x += sv.entry_w[3 * k + 0] * s;
        cs.J.y += sv.entry_w[3 * k + 1] * s;
        cs.J.z += sv.entry_w[3 * k + 2] * s;
    }
    const uint32_t mask = sv.impose_mask[m];
    cs.imposed = mask != 0u;
    for (int k = 0; k < kMaxSources; ++k) {
        if ((mask >> k) & 1u) {
            const float s = sc.s[k];
            cs.E.x += sc.E0[k][0] * s;
            cs.E.y += sc.E0[k][1] * s;
            cs.E.z += sc.E0[k][2] * s;
            cs.B.x += sc.B0[k][0] * s;
            cs.B.y += sc.B0[k][1] * s;
            cs.B.z += sc.B0[k][2] * s;
        }
    }
    return cs;
}

// Block-wide sum of three doubles (blockDim.x == kBlock), stored by thread 0 in a fixed order.
__device__ __forceinline__ void block_sum3_store(double a0, double a1, double a2, double* out) {
    __shared__ double sh[3][kBlock / 32];
    for (int off = 16; off > 0; off >>= 1) {
        a0 += __shfl_down_sync(0xffffffffu, a0, off);
        a1 += __shfl_down_sync(0xffffffffu, a1, off);
        a2 += __shfl_down_sync(0xffffffffu, a2, off);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][w] = a0;
        sh[1][w] = a1;
        sh[2][w] = a2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int k = 0; k < kBlock / 32; ++k) {
            s0 += sh[0][k];
            s1 += sh[1][k];
            s2 += sh[2][k];
        }
        out[0] = s0;
        out[1] = s1;
        out[2] = s2;
    }
}

// --- host-side launchers (one set per model) -----------------------------------------------
// Each returns the number of kernels it enqueued (errors are read with cudaGetLastError).
int mm_launch_step(const StepArgs& a, cudaStream_t st);
int mm_launch_init(const StepArgs& a, const float* E, const float* B, cudaStream_t st);
int mm_launch_fields(const StepArgs& a, FieldsOut out, cudaStream_t st);
int mm_launch_get(const StepArgs& a, float* out, cudaStream_t st);
int mm_launch_set(const StepArgs& a, const float* in, cudaStream_t st);
int mm_launch_reduce(const StepArgs& a, double* partials, int n_blocks, double* result, cudaStream_t st);

int hv_launch_step(const StepArgs& a, cudaStream_t st);
int hv_launch_init(const StepArgs& a, const float* E, const float* B, cudaStream_t st);
int hv_launch_fields(const StepArgs& a, FieldsOut out, cudaStream_t st);
int hv_launch_get(const StepArgs& a, float* out, cudaStream_t st);
int hv_launch_set(const StepArgs& a, const float* in, cudaStream_t st);
int hv_launch_reduce(const StepArgs& a, double* partials, int n_blocks, double* result, cudaStream_t st);

// Deterministic double reduction of per-block partial sums (3 values per block, fixed order).
int launch_reduce_partials(const double* partials, int n_blocks, double* result, cudaStream_t st);

}  // namespace lbm
