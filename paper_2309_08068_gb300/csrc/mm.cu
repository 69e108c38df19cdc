// Mendoza-Munoz (MM) model kernels, arXiv 2309.08068 Section II.
//
// One thread updates one cell. The 48 moving populations arrive as 12 vector pulls (one per D3Q13
// velocity; the four values of a velocity move together: a float4, or 8 bytes with 16-bit storage),
// the whole collision runs in FP32 registers, and the 12 results are stored at the cell (pull
// scheme). The ordinary update is branch-free; source and imposed cells are recomputed afterwards
// with their current and imposed fields, overwriting the ordinary result: at the end of their
// block in the single-step kernels (block_source_cells), in their tile in the two-step passes, and
// by a second small launch over the merged source-cell list in the batched kernels.
//
// Direction tables. Direction d = p*4 + (i-1) with the plane p and index i of eq.
// VelocitySetMiller: v_i^p = sqrt(2) (cos((2i-1) pi/4), sin((2i-1) pi/4)) in the xy (p = 0), xz
// (p = 1) and yz (p = 2) planes, which are the edge diagonals below. The electric vectors of eq.
// ElectromagneticVectorsMiller are e_{i0} = v_{[(i+2) mod 4]+1} / 2 and e_{i1} = v_{[i mod 4]+1} / 2
// = -e_{i0}; kMMEh holds 2 e_{i0}. The magnetic vectors b_{ij} = v_i x e_{ij} come out as -z for
// every direction of plane 0, +y for plane 1 and -x for plane 2, with b_{i1} = -b_{i0}.
//
// Because e_{i1} = -e_{i0} and b_{i1} = -b_{i0}, only the differences f_{d0} - f_{d1} enter the
// moments D' and B; the sums enter only rho_c. The collision below is written per velocity in
// terms of s = v.J/16, alpha = (eps_r/4) E.e0 + B.b0/(8 mu_r) and beta = E.e0/4 + B.b0/8:
//   f^(0)eq_{d0,d1} = s +- alpha,  f^(1)eq_{d0,d1} = s +- beta   (eq. equilibriumsMiller)
//   f' = 2 f^eq - f                                              (eq. CollisionMiller)
#include "lbm_internal.cuh"

namespace lbm {
namespace {

constexpr int kMMV[12][3] = {{1, 1, 0},  {-1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                             {1, 0, 1},  {-1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
                             {0, 1, 1},  {0, -1, 1},  {0, -1, -1}, {0, 1, -1}};
constexpr int kMMEh[12][3] = {{1, -1, 0}, {1, 1, 0},  {-1, 1, 0}, {-1, -1, 0},
                              {1, 0, -1}, {1, 0, 1},  {-1, 0, 1}, {-1, 0, -1},
                              {0, 1, -1}, {0, 1, 1},  {0, -1, 1}, {0, -1, -1}};
constexpr int kMMB[12][3] = {{0, 0, -1}, {0, 0, -1}, {0, 0, -1}, {0, 0, -1},
                             {0, 1, 0},  {0, 1, 0},  {0, 1, 0},  {0, 1, 0},
                             {-1, 0, 0}, {-1, 0, 0}, {-1, 0, 0}, {-1, 0, 0}};

// Dot product of a compile-time {-1,0,1} vector row with (x, y, z).
template <int A, int B, int C>
__device__ __forceinline__ float sdot(float x, float y, float z) {
    float s = 0.f;
    acc<A>(s, x);
    acc<B>(s, y);
    acc<C>(s, z);
    return s;
}

struct MMFields {
    float3 X;    // D' - mu0 J_ext / 4 (so that Dpp = X g)
    float3 Dpp;  // eps_r E = D (physical displacement, eps0 = 1)
    float3 E;
    float3 B;
    float3 J;
    float rho;
    float inv4mu;  // 1 / (4 mu_r)
};

// Moments of the 48 moving populations (eq. MacroscopicFieldsMiller), then E and J with ohmic
// conductivity and an external current (eqs. MacroscopicEMiller, MacorscopicCurrentMiller):
//   eps_r E = (D' - mu0 J_ext / 4) / (1 + mu0 sigma / (4 eps_r)),  J = sigma E + J_ext,  mu0 = 2.
// Position of direction d among the directions whose row of table T has a non-zero component a.
template <const int (&T)[12][3]>
constexpr int rank_in_column(int d, int a) {
    int r = 0;
    for (int k = 0; k < d; ++k) r += T[k][a] != 0;
    return r;
}

// Signed terms of one moment component, sum_d T[d][a] * x_d, summed pairwise in direction order.
// Each component of D' has 8 terms (2 e_{i0} has two non-zero entries), each component of B has 4.
template <const int (&T)[12][3], int A, int N>
__device__ __forceinline__ float moment_component(const float (&x)[12]) {
    float t[N];
    static_for<0, 12>([&](auto dc) {
        constexpr int d = decltype(dc)::value;
        if constexpr (T[d][A] != 0) {
            constexpr int r = rank_in_column<T>(d, A);
            if constexpr (T[d][A] > 0) t[r] = x[d];
            else t[r] = -x[d];
        }
    });
    return pairwise_sum<0, N>(t);
}

// eps_r E = Dpp = X g and E = Dpp / eps_r, each rounded once (__fmul_rn: never fused into a later
// sum), so that the backward step can recompute E from the recorded X and get the same bits.
__device__ __forceinline__ float3 mm_dpp(float3 X, float g) {
    return make_float3(__fmul_rn(X.x, g), __fmul_rn(X.y, g), __fmul_rn(X.z, g));
}
__device__ __forceinline__ float3 mm_e_of_dpp(float3 Dpp, float er, float inv_er) {
    return make_float3(div_rn(Dpp.x, er, inv_er), div_rn(Dpp.y, er, inv_er), div_rn(Dpp.z, er, inv_er));
}

template <bool kRho>
__device__ __forceinline__ MMFields mm_fields(const float4 (&f)[12], float rest0, const MatCoef& mat, float3 jext) {
    float de[12], db[12];
    float rho = rest0;
    static_for<0, 12>([&](auto dc) {
        constexpr int d = decltype(dc)::value;
        de[d] = f[d].x - f[d].y;
        db[d] = f[d].z - f[d].w;
        if constexpr (kRho) rho += f[d].x + f[d].y;
    });
    const float dx = moment_component<kMMEh, 0, 8>(de), dy = moment_component<kMMEh, 1, 8>(de),
                dz = moment_component<kMMEh, 2, 8>(de);
    const float bx = moment_component<kMMB, 0, 4>(db), by = moment_component<kMMB, 1, 4>(db),
                bz = moment_component<kMMB, 2, 4>(db);
    MMFields o;
    const float g = mat.c0.z;  // 1 / (1 + mu0 sigma / (4 eps_r))
    const float er = mat.c0.x, inv_er = mat.c0.y, sigma = mat.c1.x;
    o.X = make_float3(0.5f * dx - 0.5f * jext.x, 0.5f * dy - 0.5f * jext.y, 0.5f * dz - 0.5f * jext.z);
    o.Dpp = mm_dpp(o.X, g);
    o.E = mm_e_of_dpp(o.Dpp, er, inv_er);
    o.B = make_float3(bx, by, bz);
    // Explicit fused multiply-adds wherever a product is inexact, so that the result does not
    // depend on the compiler's contraction choices (the batched and single-lattice kernels inline
    // this code in different contexts and must agree bit for bit).
    o.J.x = __fmaf_rn(sigma, o.E.x, jext.x);
    o.J.y = __fmaf_rn(sigma, o.E.y, jext.y);
    o.J.z = __fmaf_rn(sigma, o.E.z, jext.z);
    o.rho = rho;
    o.inv4mu = mat.c0.w;
    return o;
}

// Pull the 12 groups of cell i from the previous step's buffer: direction d from cell i - v_d.
// 24-bit storage: the 12 planes of halves (8 B per group and cell), then the 12 planes of correction
// bytes (4 B per group and cell).
template <int S>
__device__ __forceinline__ void mm_pull(const StepArgs& a, const Neighbourhood& h, float4 (&f)[12]) {
    if constexpr (S == kF24) {
        const uint2* __restrict__ hi = static_cast<const uint2*>(a.fin);
        const unsigned* __restrict__ lo = reinterpret_cast<const unsigned*>(hi + 12 * (size_t)a.g.n);
        static_for<0, 12>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            const int src = shifted<-kMMV[d][0], -kMMV[d][1], -kMMV[d][2]>(h);
            f[d] = F24::load4(hi, lo, (size_t)d * a.g.n + src, a.inv_scale);
        });
    } else {
        const auto* __restrict__ fin = static_cast<const typename Pack4<S>::T*>(a.fin);
        static_for<0, 12>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            const int src = shifted<-kMMV[d][0], -kMMV[d][1], -kMMV[d][2]>(h);
            f[d] = Pack4<S>::load(fin + (size_t)d * a.g.n + src, a.inv_scale);
        });
    }
}

// Prefetch into L2 what the update of cell i will load: the populations mm_pull reads and the medium.
template <int S, int M>
__device__ __forceinline__ void mm_prefetch(const StepArgs& a, int i) {
    prefetch_media<M>(a.media, i);
    const auto* __restrict__ fin = static_cast<const typename Pack4<S>::T*>(a.fin);
    const Neighbourhood h = neighbourhood(a.g, i);
    static_for<0, 12>([&](auto dc) {
        constexpr int d = decltype(dc)::value;
        prefetch_l2(fin + (size_t)d * a.g.n + shifted<-kMMV[d][0], -kMMV[d][1], -kMMV[d][2]>(h));
    });
}

template <int S>
__device__ __forceinline__ void mm_put(const StepArgs& a, int d, int i, float4 v) {
    if constexpr (S == kF24) {
        uint2* __restrict__ hi = static_cast<uint2*>(a.fout);
        unsigned* __restrict__ lo = reinterpret_cast<unsigned*>(hi + 12 * (size_t)a.g.n);
        F24::store4(hi, lo, (size_t)d * a.g.n + i, v, a.scale);
    } else {
        auto* __restrict__ fout = static_cast<typename Pack4<S>::T*>(a.fout);
        fout[(size_t)d * a.g.n + i] = Pack4<S>::pack(v, a.scale);
    }
}

// Where a step reads its populations and writes its results: the context's A/B buffers.
struct MMBuffers : NoStash {
    template <int S>
    __device__ void pull(const StepArgs& a, const Neighbourhood& h, float4 (&f)[12]) const {
        mm_pull<S>(a, h, f);
    }
    template <int S>
    __device__ void put(const StepArgs& a, int d, int i, float4 v) const {
        mm_put<S>(a, d, i, v);
    }
};

// Update of cell i; m is its index in the special-cell list when kSpecial.
template <int S, int M, bool kSpecial, bool kRho, bool kRecord = false, class IO = MMBuffers>
__device__ __forceinline__ void mm_update(const StepArgs& a, int i, int m, const IO& io = IO{}) {
    const Neighbourhood h = neighbourhood(a.g, i);
    float4 f[12];
    io.template pull<S>(a, h, f);
    if constexpr (IO::kStash)  // the f^(1) halves wait in shared memory until the collision
        static_for<0, 12>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            io.stash_put(d, f[d].z, f[d].w);
        });
    const MatCoef mat = load_coef<kModelMM, M>(a.media, i, a.eps0, a.mu0);
    float rest0 = 0.f;
    if constexpr (kRho) rest0 = a.rho_in[i];
    CellSource cs;
    float3 jext = make_float3(0.f, 0.f, 0.f);
    if constexpr (kSpecial) {
        cs = cell_source(a.sv, a.sc, m);
        jext = cs.J;
    }
    const MMFields F = mm_fields<kRho>(f, rest0, mat, jext);
    static_for<0, 12>([&](auto dc) {
        constexpr int d = decltype(dc)::value;
        constexpr int v0 = kMMV[d][0], v1 = kMMV[d][1], v2 = kMMV[d][2];
        constexpr int e0 = kMMEh[d][0], e1 = kMMEh[d][1], e2 = kMMEh[d][2];
        constexpr int b0 = kMMB[d][0], b1 = kMMB[d][1], b2 = kMMB[d][2];
        const float two_s = 0.125f * sdot<v0, v1, v2>(F.J.x, F.J.y, F.J.z);
        const float bb = sdot<b0, b1, b2>(F.B.x, F.B.y, F.B.z);
        const float two_alpha = __fmaf_rn(bb, F.inv4mu, 0.25f * sdot<e0, e1, e2>(F.Dpp.x, F.Dpp.y, F.Dpp.z));
        const float two_beta = 0.25f * sdot<e0, e1, e2>(F.E.x, F.E.y, F.E.z) + 0.25f * bb;
        float4 o;
        o.x = two_s + two_alpha - f[d].x;
        o.y = two_s - two_alpha - f[d].y;
        float fz = f[d].z, fw = f[d].w;
        if constexpr (IO::kStash) io.stash_get(d, fz, fw);
        o.z = two_s + two_beta - fz;
        o.w = two_s - two_beta - fw;
        if constexpr (kSpecial) {
            if (cs.imposed) {  // Appendix B "impose fields": f' = f_eq(E_imp, B_imp, J = 0)
                const float bi = sdot<b0, b1, b2>(cs.B.x, cs.B.y, cs.B.z);
                const float ee = sdot<e0, e1, e2>(cs.E.x, cs.E.y, cs.E.z);
                const float alpha = __fmaf_rn(0.5f * bi, F.inv4mu, 0.125f * __fmul_rn(mat.c0.x, ee));
                const float beta = 0.125f * ee + 0.125f * bi;
                o = make_float4(alpha, -alpha, beta, -beta);
            }
        }
        io.template put<S>(a, d, i, o);
    });
    if constexpr (kRho) a.rho_out[i] = 2.f * F.rho - rest0;  // f_0^(0)eq = rho_c; stays in place
    if constexpr (kRecord) {  // what the adjoint of this step needs: X (E follows from it)
        if (!io.keeps_record()) return;
        const int n = a.g.n;
        a.rec[i] = F.X.x;
        a.rec[n + i] = F.X.y;
        a.rec[2 * n + i] = F.X.z;
    }
}

// 3 resident blocks for FP32 storage; 4 for 16-bit storage, whose halved bytes need more loads in
// flight per SM to reach the copy bandwidth (256^3 dipole on GB300, BF16: 0.475 against 0.497 ms
// per step at 3 blocks); 3 for 24-bit storage, whose decoding would spill at 64 registers.
// The block's source cells are recomputed at the end (block_source_cells).
template <int S, int M, bool kRho>
__global__ void __launch_bounds__(kBlock, S == kF32 || S == kF24 ? 3 : 4) mm_step_kernel(StepArgs a) {
    const int i = a.cell_begin + blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.cell_end) mm_update<S, M, false, kRho>(a, i, 0);
    block_source_cells(a.sv, blockIdx.x, [&](int c, int m) { mm_update<S, M, true, kRho>(a, c, m); });
}

// Equilibrium populations of cell x for fields E, B and J = 0 (Appendix B initialisation).
template <int S, int M>
__global__ void __launch_bounds__(kBlock) mm_init_kernel(StepArgs a, const float* __restrict__ E,
                                                         const float* __restrict__ B) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= a.g.n) return;
    const int n = a.g.n;
    const Neighbourhood h = neighbourhood(a.g, y);
    // Stored value at y for direction d is the population cell x = y + v_d pulls next step.
    static_for<0, 12>([&](auto dc) {
        constexpr int d = decltype(dc)::value;
        constexpr int e0 = kMMEh[d][0], e1 = kMMEh[d][1], e2 = kMMEh[d][2];
        constexpr int b0 = kMMB[d][0], b1 = kMMB[d][1], b2 = kMMB[d][2];
        const int x = shifted<kMMV[d][0], kMMV[d][1], kMMV[d][2]>(h);
        const MatCoef mat = load_coef<kModelMM, M>(a.media, x, a.eps0, a.mu0);
        const float ee = sdot<e0, e1, e2>(__ldg(&E[x]), __ldg(&E[n + x]), __ldg(&E[2 * n + x]));
        const float bb = sdot<b0, b1, b2>(__ldg(&B[x]), __ldg(&B[n + x]), __ldg(&B[2 * n + x]));
        const float alpha = __fmaf_rn(bb, 0.5f * mat.c0.w, 0.125f * __fmul_rn(mat.c0.x, ee));  // 0.5 / (4 mu_r)
        const float beta = 0.125f * ee + 0.125f * bb;
        mm_put<S>(a, d, y, make_float4(alpha, -alpha, beta, -beta));
    });
}

template <int S, int M, bool kSpecial>
__global__ void __launch_bounds__(kBlock) mm_fields_kernel(StepArgs a, FieldsOut out) {
    int i, m = 0;
    if constexpr (kSpecial) {
        m = blockIdx.x * blockDim.x + threadIdx.x;
        if (m >= a.sv.n_special) return;
        i = a.sv.cell[m];
    } else {
        i = blockIdx.x * blockDim.x + threadIdx.x;
        if (i >= a.g.n) return;
    }
    const int n = a.g.n;
    const Neighbourhood h = neighbourhood(a.g, i);
    float4 f[12];
    mm_pull<S>(a, h, f);
    const MatCoef mat = load_coef<kModelMM, M>(a.media, i, a.eps0, a.mu0);
    float3 jext = make_float3(0.f, 0.f, 0.f);
    if constexpr (kSpecial) jext = cell_source(a.sv, a.sc, m).J;
    const MMFields F = mm_fields<false>(f, 0.f, mat, jext);
    auto put = [&](float* p, float3 v) {
        if (p) {
            p[i] = v.x;
            p[n + i] = v.y;
            p[2 * n + i] = v.z;
        }
    };
    put(out.E, F.E);
    put(out.B, F.B);
    put(out.D, F.Dpp);  // D = eps0 eps_r E with eps0 = 1
    // H = B / (mu0 mu_r) with mu0 = 2; 1 / (2 mu_r) = 2 / (4 mu_r) exactly
    const float two_mu = 2.f * mat.c1.y, inv2mu = 2.f * mat.c0.w;
    put(out.H, make_float3(div_rn(F.B.x, two_mu, inv2mu), div_rn(F.B.y, two_mu, inv2mu),
                           div_rn(F.B.z, two_mu, inv2mu)));
    put(out.J, F.J);
}

// Canonical layout out[k * n + x]: k = r*24 + p*8 + (i-1)*2 + j = r*24 + 2d + j; 48, 49 rest.
template <int S>
__global__ void __launch_bounds__(kBlock) mm_get_kernel(StepArgs a, const float* __restrict__ rest1,
                                                        float* __restrict__ out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.g.n) return;
    const int n = a.g.n;
    const Neighbourhood h = neighbourhood(a.g, x);
    float4 f[12];
    mm_pull<S>(a, h, f);
    static_for<0, 12>([&](auto dc) {
        constexpr int d = decltype(dc)::value;
        out[(size_t)(2 * d) * n + x] = f[d].x;
        out[(size_t)(2 * d + 1) * n + x] = f[d].y;
        out[(size_t)(24 + 2 * d) * n + x] = f[d].z;
        out[(size_t)(25 + 2 * d) * n + x] = f[d].w;
    });
    out[(size_t)48 * n + x] = a.rho_in ? a.rho_in[x] : 0.f;
    out[(size_t)49 * n + x] = rest1 ? rest1[x] : 0.f;
}

template <int S>
__global__ void __launch_bounds__(kBlock) mm_set_kernel(StepArgs a, const float* __restrict__ in,
                                                        float* __restrict__ rest1) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= a.g.n) return;
    const int n = a.g.n;
    const Neighbourhood h = neighbourhood(a.g, y);
    static_for<0, 12>([&](auto dc) {
        constexpr int d = decltype(dc)::value;
        const int x = shifted<kMMV[d][0], kMMV[d][1], kMMV[d][2]>(h);
        mm_put<S>(a, d, y,
                  make_float4(in[(size_t)(2 * d) * n + x], in[(size_t)(2 * d + 1) * n + x],
                              in[(size_t)(24 + 2 * d) * n + x], in[(size_t)(25 + 2 * d) * n + x]));
    });
    if (a.rho_out) a.rho_out[y] = in[(size_t)48 * n + y];
    if (rest1) rest1[y] = in[(size_t)49 * n + y];
}

// Per-block partial sums of (1/2)(E.D + B.H), sum f^2 and rho_c over a grid-stride range of cells
// (external current taken as zero here; the special-cell pass adds the correction).
template <int S, int M, bool kRho>
__global__ void __launch_bounds__(kBlock) mm_reduce_kernel(StepArgs a, const float* __restrict__ rest1,
                                                           double* __restrict__ partials) {
    double w = 0.0, f2 = 0.0, q = 0.0;
    for (int i = a.cell_begin + blockIdx.x * blockDim.x + threadIdx.x; i < a.cell_end; i += gridDim.x * blockDim.x) {
        const Neighbourhood h = neighbourhood(a.g, i);
        float4 f[12];
        mm_pull<S>(a, h, f);
        const MatCoef mat = load_coef<kModelMM, M>(a.media, i, a.eps0, a.mu0);
        float rest0 = 0.f;
        if constexpr (kRho) rest0 = a.rho_in[i];
        const MMFields F = mm_fields<kRho>(f, rest0, mat, make_float3(0.f, 0.f, 0.f));
        const double inv2mu = 1.0 / (2.0 * (double)mat.c1.y);
        w += 0.5 * ((double)F.E.x * F.Dpp.x + (double)F.E.y * F.Dpp.y + (double)F.E.z * F.Dpp.z) +
             0.5 * inv2mu * ((double)F.B.x * F.B.x + (double)F.B.y * F.B.y + (double)F.B.z * F.B.z);
        double s = 0.0;
#pragma unroll
        for (int d = 0; d < 12; ++d)
            s += (double)f[d].x * f[d].x + (double)f[d].y * f[d].y + (double)f[d].z * f[d].z +
                 (double)f[d].w * f[d].w;
        if constexpr (kRho) {
            s += (double)rest0 * rest0;
            q += F.rho;
        }
        if (rest1) s += (double)rest1[i] * rest1[i];
        f2 += s;
    }
    block_sum3_store(w, f2, q, partials + 3 * blockIdx.x);
}

// Energy correction at source cells: (energy with J_ext) - (energy with J_ext = 0).
template <int S, int M>
__global__ void __launch_bounds__(kBlock) mm_reduce_special_kernel(StepArgs a, double* __restrict__ partials) {
    double w = 0.0;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < a.sv.n_special) {
        const int i = a.sv.cell[m];
        const Neighbourhood h = neighbourhood(a.g, i);
        float4 f[12];
        mm_pull<S>(a, h, f);
        const MatCoef mat = load_coef<kModelMM, M>(a.media, i, a.eps0, a.mu0);
        const MMFields F1 = mm_fields<false>(f, 0.f, mat, cell_source(a.sv, a.sc, m).J);
        const MMFields F0 = mm_fields<false>(f, 0.f, mat, make_float3(0.f, 0.f, 0.f));
        w = 0.5 * ((double)F1.E.x * F1.Dpp.x + (double)F1.E.y * F1.Dpp.y + (double)F1.E.z * F1.Dpp.z) -
            0.5 * ((double)F0.E.x * F0.Dpp.x + (double)F0.E.y * F0.Dpp.y + (double)F0.E.z * F0.Dpp.z);
    }
    block_sum3_store(w, 0.0, 0.0, partials + 3 * blockIdx.x);
}

// Batched step j of several lattices: each block takes tiles (lattice, first cell) in turn; with a
// grid smaller than the tile count the blocks persist and stride over the tiles.
template <int S, int BLOCK, bool kRho>
__global__ void __launch_bounds__(BLOCK, 768 / BLOCK) mm_batch_kernel(const BatchLattice* __restrict__ lat,
                                                                        const BatchTile* __restrict__ tiles,
                                                                        int n_tiles, int j) {
    for (int b = blockIdx.x; b < n_tiles; b += gridDim.x) {
        const BatchTile tile = tiles[b];
        const BatchLattice* L = &lat[tile.lattice];
        const int i = tile.begin + threadIdx.x;
        if (j >= L->steps || i >= L->base.g.n) continue;
        const StepArgs a = batch_args(L, j);
        switch (a.media_mode) {
            case kUniform: mm_update<S, kUniform, false, kRho>(a, i, 0); break;
            case kTable: mm_update<S, kTable, false, kRho>(a, i, 0); break;
            default: mm_update<S, kPerCell, false, kRho>(a, i, 0); break;
        }
    }
}

template <int S, bool kRho>
__global__ void __launch_bounds__(kBlock) mm_batch_special_kernel(const BatchLattice* __restrict__ lat,
                                                                  const BatchTile* __restrict__ tiles, int j) {
    const BatchTile tile = tiles[blockIdx.x];
    const BatchLattice* L = &lat[tile.lattice];
    const int m = tile.begin + threadIdx.x;
    if (j >= L->steps || m >= L->base.sv.n_special) return;
    StepArgs a = batch_args(L, j);
    batch_sources(L, j, a);
    const int i = a.sv.cell[m];
    switch (a.media_mode) {
        case kUniform: mm_update<S, kUniform, true, kRho>(a, i, m); break;
        case kTable: mm_update<S, kTable, true, kRho>(a, i, m); break;
        default: mm_update<S, kPerCell, true, kRho>(a, i, m); break;
    }
}

template <int M, bool kRho>
__global__ void __launch_bounds__(kBlock, 3) mm_record_kernel(StepArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.g.n) mm_update<kF32, M, false, kRho, true>(a, i, 0);
    block_source_cells(a.sv, blockIdx.x, [&](int c, int m) { mm_update<kF32, M, true, kRho, true>(a, c, m); });
}

// ---------------------------------------------------------------------------------------------
// Two steps per pass (see FusedArgs). Phase A reads the A/B buffer once (streaming loads that L2
// may evict first) and writes the intermediate plane; phase B pulls from the intermediate planes
// (L2 loads: they were written by other blocks of this launch) and writes the other A/B buffer
// once (streaming stores). The arithmetic is mm_update's, so the pair of steps gives the same
// bits as two single steps.
template <int S>
struct MMToRing : FusedStash {
    using T = typename Pack4<S>::T;
    T* plane;  // slot of this cell's plane
    int base;  // first cell of the plane
    int nxy;
    template <int S2>
    __device__ void pull(const StepArgs& a, const Neighbourhood& h, float4 (&f)[12]) const {
        const T* __restrict__ fin = static_cast<const T*>(a.fin);
        static_for<0, 12>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            const int src = shifted<-kMMV[d][0], -kMMV[d][1], -kMMV[d][2]>(h);
            f[d] = Pack4<S>::unpack(__ldcs(fin + (size_t)d * a.g.n + src), a.inv_scale);
        });
    }
    template <int S2>
    __device__ void put(const StepArgs& a, int d, int i, float4 v) const {
        __stcg(plane + (size_t)d * nxy + (i - base), Pack4<S>::pack(v, a.scale));
    }
};

template <int S>
struct MMFromRing : FusedStash {
    using T = typename Pack4<S>::T;
    const T* plane[3];  // slots of planes z - 1, z, z + 1
    int nxy;
    template <int S2>
    __device__ void pull(const StepArgs& a, const Neighbourhood& h, float4 (&f)[12]) const {
        static_for<0, 12>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            constexpr int sx = -kMMV[d][0], sy = -kMMV[d][1], sz = -kMMV[d][2];
            const T* src = plane[sz + 1] + (size_t)d * nxy + h.xo[sx + 1] + h.yo[sy + 1];
            f[d] = Pack4<S>::unpack(__ldcg(src), a.inv_scale);
        });
    }
    template <int S2>
    __device__ void put(const StepArgs& a, int d, int i, float4 v) const {
        T* __restrict__ fout = static_cast<T*>(a.fout);
        __stcs(fout + (size_t)d * a.g.n + i, Pack4<S>::pack(v, a.scale));
    }
};

template <int S, int M>
__global__ void __launch_bounds__(kFusedThreads, 3) mm_fused2_kernel(StepArgs aA, StepArgs aB, FusedArgs F) {
    using T = typename Pack4<S>::T;
    __shared__ float2 s_stash[12 * kBlock];  // the f^(1) halves, [velocity][compute thread]
    const unsigned stash = fused_stash_slot(s_stash);
    const int nz = aA.g.nz, nxy = aA.g.nx * aA.g.ny;
    auto slot = [&](int p) -> T* {
        if (p == 0) return static_cast<T*>(F.lo);
        if (p == nz - 1) return static_cast<T*>(F.hi);
        return static_cast<T*>(F.ring) + (size_t)(p % F.R) * 12 * nxy;
    };
    auto describe = [&](const FusedItem& it, FusedDesc& d) {
        if (it.type == kPhaseA) {
            d.ptr[0] = slot(it.plane);
        } else {
            d.ptr[0] = slot((it.plane + nz - 1) % nz);
            d.ptr[1] = slot(it.plane);
            d.ptr[2] = slot((it.plane + 1) % nz);
        }
    };
    fused_loop(F, aA.g.nx, nxy, nz, describe, [&](const FusedDesc& d) {
        const int j = d.j, base = d.plane * nxy;
        if (d.type == kPhaseA) {
            const MMToRing<S> io{{stash}, static_cast<T*>(d.ptr[0]), base, nxy};
            const int end = min(base + (j + 1) * F.tile_cells, base + nxy);
            for (int i = base + j * F.tile_cells + threadIdx.x; i < end; i += kBlock)
                mm_update<S, M, false, false, false>(aA, i, 0, io);
            if (d.s_hi > d.s_lo) {  // the tile's source cells replace their ordinary update
                named_sync(kComputeBarrier, kBlock);
                for (int m = d.s_lo + threadIdx.x; m < d.s_hi; m += kBlock)
                    mm_update<S, M, true, false, false>(aA, aA.sv.cell[m], m, io);
            }
        } else {
            const MMFromRing<S> io{{stash},
                                   {static_cast<const T*>(d.ptr[0]), static_cast<const T*>(d.ptr[1]),
                                    static_cast<const T*>(d.ptr[2])},
                                   nxy};
            const int end = min(base + (j + 1) * F.tile_cells, base + nxy);
            for (int i = base + j * F.tile_cells + threadIdx.x; i < end; i += kBlock)
                mm_update<S, M, false, false, false>(aB, i, 0, io);
            if (d.s_hi > d.s_lo) {  // the tile's source cells replace their ordinary update
                named_sync(kComputeBarrier, kBlock);
                for (int m = d.s_lo + threadIdx.x; m < d.s_hi; m += kBlock)
                    mm_update<S, M, true, false, false>(aB, aB.sv.cell[m], m, io);
            }
        }
    });
}

// ---------------------------------------------------------------------------------------------
// Two steps per pass over shared-memory tiles (see TileArgs). Directions by v_z: class 0 (in-plane,
// d = 0..3), class 1 (v_z = +1: d = 4, 5, 8, 9), class 2 (v_z = -1: d = 6, 7, 10, 11); four
// directions per class.
__host__ __device__ constexpr int mm_zclass(int d) { return d < 4 ? 0 : (((d >> 1) & 1) ? 2 : 1); }
__host__ __device__ constexpr int mm_zrank(int d) { return d < 4 ? d : (d & 1) + (d >= 8 ? 2 : 0); }
static_assert(mm_zclass(4) == 1 && mm_zclass(9) == 1 && mm_zclass(6) == 2 && mm_zclass(11) == 2 &&
                  mm_zrank(8) == 2 && mm_zrank(10) == 2 && mm_zrank(7) == 1,
              "v_z classes of the D3Q13 velocity table");

// Six slots of 4 directions x kTileThreads cells: slot 0 the class-2 directions of the newest
// plane, slots 1-2 class 0 of the last two planes, slots 3-5 class 1 of the last three.
template <int S>
struct MMTile {
    using T = typename Pack4<S>::T;
    static constexpr size_t kBytes = 6 * 4 * kTileThreads * sizeof(T);
    T* base;
    __device__ T* slot(int cls, int p) const {  // plane p >= -1
        const int s = cls == 2 ? 0 : (cls == 0 ? 1 + (p + 3) % 2 : 3 + (p + 3) % 3);
        return base + (size_t)s * 4 * kTileThreads;
    }
};

// Phase A: pulls from the A/B buffer, results into the tile's slots of plane p.
template <int S>
struct MMToTile : NoStash {
    using T = typename Pack4<S>::T;
    T* dst[3];  // slots of plane p, by class
    int local;  // extended-tile position of the cell
    bool own;   // a cell of the block's own tile and planes: a recording pass writes its record
    __device__ bool keeps_record() const { return own; }
    template <int S2>
    __device__ void pull(const StepArgs& a, const Neighbourhood& h, float4 (&f)[12]) const {
        mm_pull<S>(a, h, f);
    }
    template <int S2>
    __device__ void put(const StepArgs& a, int d, int, float4 v) const {
        dst[mm_zclass(d)][mm_zrank(d) * kTileThreads + local] = Pack4<S>::pack(v, a.scale);
    }
};

// Phase B: pulls from the tile (class 0 from plane q, class 1 from q - 1, class 2 from q + 1),
// results into the other A/B buffer.
template <int S>
struct MMFromTile : NoStash {
    using T = typename Pack4<S>::T;
    const T* src[3];
    int local;
    template <int S2>
    __device__ void pull(const StepArgs& a, const Neighbourhood&, float4 (&f)[12]) const {
        static_for<0, 12>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            static_assert(kMMV[d][2] == (mm_zclass(d) == 0 ? 0 : (mm_zclass(d) == 1 ? 1 : -1)), "class of d");
            constexpr int off = mm_zrank(d) * kTileThreads - (kMMV[d][0] + kMMV[d][1] * kTileEX);
            f[d] = Pack4<S>::unpack(src[mm_zclass(d)][off + local], a.inv_scale);
        });
    }
    template <int S2>
    __device__ void put(const StepArgs& a, int d, int i, float4 v) const {
        T* __restrict__ fout = static_cast<T*>(a.fout);
        __stcs(fout + (size_t)d * a.g.n + i, Pack4<S>::pack(v, a.scale));
    }
};

// kRecord: both steps also write the adjoint's per-cell records (aA.rec, aB.rec), each cell's once,
// by the block that owns it.
template <int S, int M, bool kRecord = false>
__global__ void __launch_bounds__(kTileThreads, S == kF32 ? 2 : 3) mm_tile2_kernel(StepArgs aA, StepArgs aB,
                                                                                    TileArgs T) {
    using TT = typename Pack4<S>::T;
    extern __shared__ __align__(16) unsigned char mm_tile_smem[];
    const MMTile<S> tile{reinterpret_cast<TT*>(mm_tile_smem)};
    const int nz = aA.g.nz, nxy = aA.g.nx * aA.g.ny;
    const TileCell c = tile_cell(aA.g, T);
    const int* off = T.entry_off + (size_t)c.tile * nz;
    for (int p = c.z0 - 1; p <= c.z1; ++p) {
        const int pz = tile_wrap(p, nz);
        // The next plane's phase-A inputs, fetched into L2 while this plane is stepped: a plane's
        // loads are otherwise a DRAM round trip that two blocks per SM cannot hide.
        if (p < c.z1) mm_prefetch<S, M>(aA, tile_wrap(p + 1, nz) * nxy + c.cxy);
        {  // phase A: step t of the extended tile's cells of plane pz
            const bool own_plane = p >= c.z0 && p < c.z1;
            const MMToTile<S> io{{}, {tile.slot(0, p), tile.slot(1, p), tile.slot(2, p)}, (int)threadIdx.x,
                                 own_plane && c.core};
            mm_update<S, M, false, false, kRecord>(aA, pz * nxy + c.cxy, 0, io);
            const int lo = off[pz], hi = off[pz + 1];
            if (hi > lo) {  // the source cells among them replace their ordinary update
                __syncthreads();
                for (int k = lo + threadIdx.x; k < hi; k += kTileThreads) {
                    const int2 e = T.entries[k];
                    const MMToTile<S> sio{{}, {io.dst[0], io.dst[1], io.dst[2]}, e.y,
                                          own_plane && tile_core(e.y, c.bx, c.by, aA.g.nx, aA.g.ny)};
                    mm_update<S, M, true, false, kRecord>(aA, aA.sv.cell[e.x], e.x, sio);
                }
            }
        }
        __syncthreads();
        if (p > c.z0) {  // phase B: step t + 1 of the tile's own cells of plane q = p - 1
            const int q = p - 1;
            const MMFromTile<S> io{{}, {tile.slot(0, q), tile.slot(1, q - 1), tile.slot(2, q + 1)}, (int)threadIdx.x};
            if (c.core) mm_update<S, M, false, false, kRecord>(aB, q * nxy + c.cxy, 0, io);
            const int lo = off[q], hi = off[q + 1];
            if (hi > lo) {
                __syncthreads();
                for (int k = lo + threadIdx.x; k < hi; k += kTileThreads) {
                    const int2 e = T.entries[k];
                    if (!tile_core(e.y, c.bx, c.by, aA.g.nx, aA.g.ny)) continue;
                    const MMFromTile<S> sio{{}, {io.src[0], io.src[1], io.src[2]}, e.y};
                    mm_update<S, M, true, false, kRecord>(aB, aB.sv.cell[e.x], e.x, sio);
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------------
// Adjoint of one MM step. With per-velocity adjoints (a0^, a1^, c0^, c1^) of the post-collision
// values, the transpose of eq. CollisionMiller through eq. equilibriumsMiller is
//   adjoint of 2s_d = a0^ + a1^ + c0^ + c1^,  of 2 alpha_d = a0^ - a1^,  of 2 beta_d = c0^ - c1^,
//   gJ = sum_d (2s_d)^ v_d / 8,   gE = sum_d (2 beta_d)^ e_d / 2 + sigma gJ   (e_d = e_{d0}, e_h = 2 e_d),
//   gB = sum_d [(2 alpha_d)^ / (4 mu_r) + (2 beta_d)^ / 4] b_d,
//   gDpp = sum_d (2 alpha_d)^ e_d / 2 + gE / eps_r   (E = Dpp / eps_r),   gX = g gDpp   (Dpp = X g),
//   D' = sum_d (f_d0 - f_d1) e_d  ->  nu(f_d0) = e_d . gX - a0^,  nu(f_d1) = -e_d . gX - a1^,
//   B  = sum_d (f'_d0 - f'_d1) b_d ->  nu(c0) = b_d . gB - c0^,  nu(c1) = -b_d . gB - c1^,
// and the parameter derivatives (g = 1 / (1 + mu0 sigma / (4 eps_r)), mu0 = 2):
//   dL/d eps_r += -gE . E / eps_r + gDpp . X * g^2 sigma / (2 eps_r^2),
//   dL/d sigma += gJ . E - gDpp . X * g^2 / (2 eps_r).
// Imposed cells output f_eq(E_imp, B_imp, 0): nothing flows back to f, and
// d alpha_d / d eps_r = e_h . E_imp / 8. The plane loss |E|^2 adds 2E to gE.
// Where a backward step reads lambda and writes nu^n, and what it does with the cell's loss and
// gradient terms: the single-step kernels read nu^{n+1} from the adjoint buffer, write nu^n back to
// one, and add the gradient terms to the per-cell sums in memory.
struct MMAdjGlobal {
    __device__ bool counts() const { return true; }  // the cell's loss and gradient terms count here
    __device__ void lam(const AdjointArgs& A, const Neighbourhood& h, float4 (&lam)[12]) const {
        const int n = A.a.g.n;
        static_for<0, 12>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            const int dst = shifted<kMMV[d][0], kMMV[d][1], kMMV[d][2]>(h);
            lam[d] = __ldg(static_cast<const float4*>(A.nu_in) + (size_t)d * n + dst);
        });
    }
    __device__ void put_nu(const AdjointArgs& A, int d, int i, float4 o) const {
        static_cast<float4*>(A.nu_out)[(size_t)d * A.a.g.n + i] = o;
    }
    __device__ void grad_load(const AdjointArgs& A, int i, float& ge, float& gs) const {
        ge = __ldg(&A.grad_eps[i]);
        if (A.grad_sigma) gs = __ldg(&A.grad_sigma[i]);
    }
    __device__ void grad_store(const AdjointArgs& A, int i, float ge, float gs) const {
        A.grad_eps[i] = ge;
        if (A.grad_sigma) A.grad_sigma[i] = gs;
    }
};

template <int M, bool kSpecial, bool kTerminal, class IO = MMAdjGlobal>
__device__ __forceinline__ void mm_adjoint_cell(const AdjointArgs& A, int i, int m, const IO& io = IO{}) {
    const StepArgs& a = A.a;
    const int n = a.g.n;
    const Neighbourhood h = neighbourhood(a.g, i);
    const MatCoef mat = load_coef<kModelMM, M>(a.media, i, a.eps0, a.mu0);
    CellSource cs;
    bool imposed = false;
    if constexpr (kSpecial) {
        cs = cell_source(a.sv, a.sc, m);
        imposed = cs.imposed;
    }
    // Every load is issued up front: the source-cell mask of the main launch only gates the stores,
    // so it adds no round trip before the others.
    const bool skip = !kSpecial && !kTerminal && A.special_mask[i] != 0;
    const bool counts = io.counts();
    float geps_old = 0.f, gsig_old = 0.f;
    if (counts) io.grad_load(A, i, geps_old, gsig_old);
    // E and X of f^n: X from the forward step's record (E recomputed from it), or (terminal) the final state
    float3 E, X;
    if constexpr (kTerminal) {
        float4 f[12];
        mm_pull<kF32>(a, h, f);
        const MMFields F = mm_fields<false>(f, 0.f, mat, make_float3(0.f, 0.f, 0.f));
        E = F.E;
        X = F.X;
    } else {
        X = make_float3(__ldg(&a.rec[i]), __ldg(&a.rec[n + i]), __ldg(&a.rec[2 * n + i]));
        E = mm_e_of_dpp(mm_dpp(X, mat.c0.z), mat.c0.x, mat.c0.y);  // as the forward step computed it
    }
    struct {
        float3 E, X;
    } F{E, X};
    const float inv_er = mat.c0.y, g = mat.c0.z, inv4mu = mat.c0.w, sigma = mat.c1.x;
    float4 lam[12];
    if constexpr (kTerminal) {
        static_for<0, 12>([&](auto dc) { lam[decltype(dc)::value] = make_float4(0.f, 0.f, 0.f, 0.f); });
    } else {
        io.lam(A, h, lam);
    }
    float gJx = 0.f, gJy = 0.f, gJz = 0.f, gAx = 0.f, gAy = 0.f, gAz = 0.f, gEx = 0.f, gEy = 0.f, gEz = 0.f;
    float gBx = 0.f, gBy = 0.f, gBz = 0.f, geps_imposed = 0.f;
    if (!imposed) {
        static_for<0, 12>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            const float s2 = (lam[d].x + lam[d].y) + (lam[d].z + lam[d].w);
            const float a2 = lam[d].x - lam[d].y, b2 = lam[d].z - lam[d].w;
            acc<kMMV[d][0]>(gJx, s2);
            acc<kMMV[d][1]>(gJy, s2);
            acc<kMMV[d][2]>(gJz, s2);
            acc<kMMEh[d][0]>(gAx, a2);
            acc<kMMEh[d][1]>(gAy, a2);
            acc<kMMEh[d][2]>(gAz, a2);
            acc<kMMEh[d][0]>(gEx, b2);
            acc<kMMEh[d][1]>(gEy, b2);
            acc<kMMEh[d][2]>(gEz, b2);
            const float bcoef = __fmaf_rn(a2, inv4mu, 0.25f * b2);
            acc<kMMB[d][0]>(gBx, bcoef);
            acc<kMMB[d][1]>(gBy, bcoef);
            acc<kMMB[d][2]>(gBz, bcoef);
        });
        gJx *= 0.125f; gJy *= 0.125f; gJz *= 0.125f;
        gEx = __fmaf_rn(sigma, gJx, 0.25f * gEx);
        gEy = __fmaf_rn(sigma, gJy, 0.25f * gEy);
        gEz = __fmaf_rn(sigma, gJz, 0.25f * gEz);
    } else if constexpr (kSpecial) {
        static_for<0, 12>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            const float ee = sdot<kMMEh[d][0], kMMEh[d][1], kMMEh[d][2]>(cs.E.x, cs.E.y, cs.E.z);
            geps_imposed = __fmaf_rn(lam[d].x - lam[d].y, 0.125f * ee, geps_imposed);
        });
    }
    if (A.loss_active && in_plane(h, a.g, A.plane_axis, A.plane_index)) {  // |E|^2 of time n
        gEx = __fmaf_rn(2.f, F.E.x, gEx);
        gEy = __fmaf_rn(2.f, F.E.y, gEy);
        gEz = __fmaf_rn(2.f, F.E.z, gEz);
        if (counts) add_plane_loss<kTerminal>(A, h, F.E);
    }
    const float gDx = __fmaf_rn(gEx, inv_er, 0.25f * gAx), gDy = __fmaf_rn(gEy, inv_er, 0.25f * gAy),
                gDz = __fmaf_rn(gEz, inv_er, 0.25f * gAz);
    // __fmul_rn: the products must not fuse into the sums below differently in different kernels
    const float gXx = __fmul_rn(g, gDx), gXy = __fmul_rn(g, gDy), gXz = __fmul_rn(g, gDz);
    if (skip) return;  // a source cell: the source-cell pass writes it
    static_for<0, 12>([&](auto dc) {
        constexpr int d = decltype(dc)::value;
        const float gde = 0.5f * sdot<kMMEh[d][0], kMMEh[d][1], kMMEh[d][2]>(gXx, gXy, gXz);
        const float gdb = sdot<kMMB[d][0], kMMB[d][1], kMMB[d][2]>(gBx, gBy, gBz);
        float4 o;
        if (imposed) o = make_float4(gde, -gde, gdb, -gdb);
        else o = make_float4(gde - lam[d].x, -gde - lam[d].y, gdb - lam[d].z, -gdb - lam[d].w);
        io.put_nu(A, d, i, o);
    });
    if (!counts) return;
    // Explicit fused multiply-adds wherever a product meets an addition: the single-step and the
    // tiled backward kernels inline this code in different contexts and must agree bit for bit.
    const float gEdotE = __fmaf_rn(gEz, F.E.z, __fmaf_rn(gEy, F.E.y, __fmul_rn(gEx, F.E.x)));
    const float gDdotX = __fmaf_rn(gDz, F.X.z, __fmaf_rn(gDy, F.X.y, __fmul_rn(gDx, F.X.x)));
    const float gJdotE = __fmaf_rn(gJz, F.E.z, __fmaf_rn(gJy, F.E.y, __fmul_rn(gJx, F.E.x)));
    const float gg = g * g * inv_er;
    float deps = __fmaf_rn(-gEdotE, inv_er, geps_imposed);
    deps = __fmaf_rn(gDdotX, gg * 0.5f * sigma * inv_er, deps);
    const float dsig = __fmaf_rn(-gDdotX, 0.5f * gg, gJdotE);
    io.grad_store(A, i, geps_old + deps, gsig_old + dsig);
}

// Two backward steps per pass over shared-memory tiles, the mirror of mm_tile2_kernel: phase A' takes
// nu^{n+1} from memory to nu^n of the extended cells of plane p (into the tile), phase B' takes nu^n
// from the tile to nu^{n-1} of the tile's own cells of plane p - 1 (into memory). A backward step
// pulls lambda_d(x) = nu_d(x + v_d), so phase B' reads the v_z = +1 directions from plane q + 1, the
// newest: the v_z classes swap roles against the forward pass. A cell's loss and gradient terms
// count once, in its own tile and chunk; its two gradient terms are added in registers in the order
// of two single steps (the sum after step n, then step n - 1), so the sums are the same bits.
__device__ __forceinline__ int mm_adj_class(int d) {
    const int c = mm_zclass(d);
    return c == 0 ? 0 : (c == 1 ? 2 : 1);  // v_z = +1: read by the very next phase B'
}

struct MMAdjTileA : MMAdjGlobal {
    float4* dst[3];  // tile slots of plane p, by adjoint class
    int local;
    bool count, carry;  // carry: keep the gradient sums in registers for phase B'
    mutable float ge_out = 0.f, gs_out = 0.f;
    __device__ bool counts() const { return count; }
    __device__ void put_nu(const AdjointArgs&, int d, int, float4 o) const {
        dst[mm_adj_class(d)][mm_zrank(d) * kTileThreads + local] = o;
    }
    __device__ void grad_store(const AdjointArgs& A, int i, float ge, float gs) const {
        if (carry) {
            ge_out = ge;
            gs_out = gs;
        } else {
            MMAdjGlobal::grad_store(A, i, ge, gs);
        }
    }
};

struct MMAdjTileB : MMAdjGlobal {
    const float4* src[3];  // tile slots by adjoint class: plane q (0), q - 1 (1), q + 1 (2)
    int local;
    bool carry;
    float ge_in, gs_in;
    __device__ void lam(const AdjointArgs&, const Neighbourhood&, float4 (&lam)[12]) const {
        static_for<0, 12>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            constexpr int off = mm_zrank(d) * kTileThreads + (kMMV[d][0] + kMMV[d][1] * kTileEX);
            lam[d] = src[mm_adj_class(d)][off + local];
        });
    }
    __device__ void grad_load(const AdjointArgs& A, int i, float& ge, float& gs) const {
        if (carry) {
            ge = ge_in;
            gs = gs_in;
        } else {
            MMAdjGlobal::grad_load(A, i, ge, gs);
        }
    }
};

// Prefetch into L2 what phase A' of cell i loads (nu^{n+1} pushed from x + v_d, the record, the
// medium, the source-cell mask, the gradient sums) and the record phase B' of cell i reads a plane later.
template <int M>
__device__ __forceinline__ void mm_adjoint_prefetch(const AdjointArgs& A1, const AdjointArgs& A2, int i) {
    const int n = A1.a.g.n;
    const Neighbourhood h = neighbourhood(A1.a.g, i);
    static_for<0, 12>([&](auto dc) {
        constexpr int d = decltype(dc)::value;
        prefetch_l2(static_cast<const float4*>(A1.nu_in) + (size_t)d * n + shifted<kMMV[d][0], kMMV[d][1], kMMV[d][2]>(h));
    });
    static_for<0, kRecordFloatsMM>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        prefetch_l2(&A1.a.rec[(size_t)k * n + i]);
        prefetch_l2(&A2.a.rec[(size_t)k * n + i]);
    });
    prefetch_media<M>(A1.a.media, i);
    prefetch_l2(&A1.special_mask[i]);
    prefetch_l2(&A1.grad_eps[i]);
    if (A1.grad_sigma) prefetch_l2(&A1.grad_sigma[i]);
}

template <int M>
__global__ void __launch_bounds__(kTileThreads, 2) mm_adjoint2_kernel(AdjointArgs A1, AdjointArgs A2, TileArgs T) {
    extern __shared__ __align__(16) unsigned char mm_adj_smem[];
    const MMTile<kF32> tile{reinterpret_cast<float4*>(mm_adj_smem)};
    const int nz = A1.a.g.nz, nxy = A1.a.g.nx * A1.a.g.ny;
    const TileCell c = tile_cell(A1.a.g, T);
    const int* off = T.entry_off + (size_t)c.tile * nz;
    float carry_ge = 0.f, carry_gs = 0.f;  // the sums of this thread's cell of plane p - 1 after phase A'
    for (int p = c.z0 - 1; p <= c.z1; ++p) {
        const int pz = tile_wrap(p, nz);
        const bool own = p >= c.z0 && p < c.z1;
        float next_ge = 0.f, next_gs = 0.f;
        if (p < c.z1) mm_adjoint_prefetch<M>(A1, A2, tile_wrap(p + 1, nz) * nxy + c.cxy);  // as in mm_tile2_kernel
        {  // phase A': the first backward step (A1) of the extended cells of plane pz
            const MMAdjTileA io{{}, {tile.slot(0, p), tile.slot(1, p), tile.slot(2, p)}, (int)threadIdx.x,
                                c.core && own, true};
            mm_adjoint_cell<M, false, false>(A1, pz * nxy + c.cxy, 0, io);
            next_ge = io.ge_out;
            next_gs = io.gs_out;
            const int lo = off[pz], hi = off[pz + 1];
            if (hi > lo) {  // source cells: their own pass, gradient sums in memory
                __syncthreads();
                for (int k = lo + threadIdx.x; k < hi; k += kTileThreads) {
                    const int2 e = T.entries[k];
                    const MMAdjTileA sio{{}, {io.dst[0], io.dst[1], io.dst[2]}, e.y,
                                         own && tile_core(e.y, c.bx, c.by, A1.a.g.nx, A1.a.g.ny), false};
                    mm_adjoint_cell<M, true, false>(A1, A1.a.sv.cell[e.x], e.x, sio);
                }
            }
        }
        __syncthreads();
        if (p > c.z0) {  // phase B': the second backward step (A2) of the tile's own cells of plane q
            const int q = p - 1;
            const MMAdjTileB io{{}, {tile.slot(0, q), tile.slot(1, q - 1), tile.slot(2, q + 1)}, (int)threadIdx.x,
                                true, carry_ge, carry_gs};
            if (c.core) mm_adjoint_cell<M, false, false>(A2, q * nxy + c.cxy, 0, io);
            const int lo = off[q], hi = off[q + 1];
            if (hi > lo) {
                __syncthreads();
                for (int k = lo + threadIdx.x; k < hi; k += kTileThreads) {
                    const int2 e = T.entries[k];
                    if (!tile_core(e.y, c.bx, c.by, A1.a.g.nx, A1.a.g.ny)) continue;
                    const MMAdjTileB sio{{}, {io.src[0], io.src[1], io.src[2]}, e.y, false, 0.f, 0.f};
                    mm_adjoint_cell<M, true, false>(A2, A2.a.sv.cell[e.x], e.x, sio);
                }
            }
        }
        __syncthreads();
        carry_ge = next_ge;
        carry_gs = next_gs;
    }
}

// Source cells (skipped by the ordinary update through the mask) are stepped back at the end of
// their block (block_source_cells).
template <int M>
__global__ void __launch_bounds__(kBlock, 3) mm_adjoint_kernel(AdjointArgs A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < A.a.g.n) mm_adjoint_cell<M, false, false>(A, i, 0);
    block_source_cells(A.a.sv, blockIdx.x, [&](int c, int m) { mm_adjoint_cell<M, true, false>(A, c, m); });
}

template <int M>
__global__ void __launch_bounds__(kBlock) mm_adjoint_terminal_kernel(AdjointArgs A, int n_plane) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_plane) return;
    mm_adjoint_cell<M, false, true>(A, plane_cell(A.a.g, A.plane_axis, A.plane_index, k), 0);
}

}  // namespace

int mm_launch_step(const StepArgs& a, cudaStream_t st) {
    const bool rho = a.rho_in != nullptr;
    int launched = 0;
    with_storage(a.storage, [&](auto sc) {
        with_media(a.media_mode, [&](auto mc) {
            constexpr int S = decltype(sc)::value, M = decltype(mc)::value;
            const int nb = blocks_for(a.cell_end - a.cell_begin);
            if (rho) mm_step_kernel<S, M, true><<<nb, kBlock, 0, st>>>(a);
            else mm_step_kernel<S, M, false><<<nb, kBlock, 0, st>>>(a);
            launched = 1;
        });
    });
    return launched;
}

int mm_launch_init(const StepArgs& a, const float* E, const float* B, cudaStream_t st) {
    with_storage(a.storage, [&](auto sc) {
        with_media(a.media_mode, [&](auto mc) {
            constexpr int S = decltype(sc)::value, M = decltype(mc)::value;
            mm_init_kernel<S, M><<<blocks_for(a.g.n), kBlock, 0, st>>>(a, E, B);
        });
    });
    return 1;
}

int mm_launch_fields(const StepArgs& a, FieldsOut out, cudaStream_t st) {
    int launched = 0;
    with_storage(a.storage, [&](auto sc) {
        with_media(a.media_mode, [&](auto mc) {
            constexpr int S = decltype(sc)::value, M = decltype(mc)::value;
            mm_fields_kernel<S, M, false><<<blocks_for(a.g.n), kBlock, 0, st>>>(a, out);
            launched = 1;
            if (a.sv.n_special > 0) {
                mm_fields_kernel<S, M, true><<<blocks_for(a.sv.n_special), kBlock, 0, st>>>(a, out);
                launched = 2;
            }
        });
    });
    return launched;
}

int mm_launch_get(const StepArgs& a, float* out, cudaStream_t st) {
    with_storage(a.storage, [&](auto sc) {
        constexpr int S = decltype(sc)::value;
        mm_get_kernel<S><<<blocks_for(a.g.n), kBlock, 0, st>>>(a, static_cast<const float*>(a.fin2), out);
    });
    return 1;
}

int mm_launch_set(const StepArgs& a, const float* in, cudaStream_t st) {
    with_storage(a.storage, [&](auto sc) {
        constexpr int S = decltype(sc)::value;
        mm_set_kernel<S><<<blocks_for(a.g.n), kBlock, 0, st>>>(a, in, static_cast<float*>(a.fout2));
    });
    return 1;
}

int mm_launch_reduce(const StepArgs& a, double* partials, int n_blocks, double* result, cudaStream_t st) {
    const bool rho = a.rho_in != nullptr;
    const float* rest1 = static_cast<const float*>(a.fin2);
    int total = n_blocks, launched = 1;
    with_storage(a.storage, [&](auto sc) {
        with_media(a.media_mode, [&](auto mc) {
            constexpr int S = decltype(sc)::value, M = decltype(mc)::value;
            if (rho) mm_reduce_kernel<S, M, true><<<n_blocks, kBlock, 0, st>>>(a, rest1, partials);
            else mm_reduce_kernel<S, M, false><<<n_blocks, kBlock, 0, st>>>(a, rest1, partials);
            if (a.sv.n_special > 0) {
                const int ns = blocks_for(a.sv.n_special);
                mm_reduce_special_kernel<S, M><<<ns, kBlock, 0, st>>>(a, partials + 3 * n_blocks);
                total += ns;
                ++launched;
            }
        });
    });
    return launched + launch_reduce_partials(partials, total, result, st);
}

int mm_launch_batch_step(const BatchLaunch& b, int j, int n_tiles, int n_stiles, cudaStream_t st) {
    int launched = 0;
    with_storage(b.storage, [&](auto sc) {
        constexpr int S = decltype(sc)::value;
        if (n_tiles > 0) {
            const int grid = b.grid_cap > 0 ? (n_tiles < b.grid_cap ? n_tiles : b.grid_cap) : n_tiles;
            if (b.block == 128) {
                if (b.rho) mm_batch_kernel<S, 128, true><<<grid, 128, 0, st>>>(b.lat, b.tiles, n_tiles, j);
                else mm_batch_kernel<S, 128, false><<<grid, 128, 0, st>>>(b.lat, b.tiles, n_tiles, j);
            } else {
                if (b.rho) mm_batch_kernel<S, 256, true><<<grid, 256, 0, st>>>(b.lat, b.tiles, n_tiles, j);
                else mm_batch_kernel<S, 256, false><<<grid, 256, 0, st>>>(b.lat, b.tiles, n_tiles, j);
            }
            ++launched;
        }
        if (n_stiles > 0) {
            if (b.rho) mm_batch_special_kernel<S, true><<<n_stiles, kBlock, 0, st>>>(b.lat, b.stiles, j);
            else mm_batch_special_kernel<S, false><<<n_stiles, kBlock, 0, st>>>(b.lat, b.stiles, j);
            ++launched;
        }
    });
    return launched;
}

int mm_batch_occupancy(int storage, int block, bool rho) {
    int blocks = 0;
    with_storage(storage, [&](auto sc) {
        constexpr int S = decltype(sc)::value;
        if (block == 128)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &blocks, rho ? mm_batch_kernel<S, 128, true> : mm_batch_kernel<S, 128, false>, 128, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &blocks, rho ? mm_batch_kernel<S, 256, true> : mm_batch_kernel<S, 256, false>, 256, 0);
    });
    return blocks;
}

int mm_launch_adjoint(const AdjointArgs& A, cudaStream_t st) {
    int launched = 0;
    with_media(A.a.media_mode, [&](auto mc) {
        constexpr int M = decltype(mc)::value;
        mm_adjoint_kernel<M><<<blocks_for(A.a.g.n), kBlock, 0, st>>>(A);
        launched = 1;
    });
    return launched;
}

int mm_launch_adjoint2(const AdjointArgs& A1, const AdjointArgs& A2, const TileArgs& T, cudaStream_t st) {
    const dim3 grid(T.tiles_x * T.tiles_y, (A1.a.g.nz + T.chunk - 1) / T.chunk);
    with_media(A1.a.media_mode, [&](auto mc) {
        constexpr int M = decltype(mc)::value;
        static bool done = false;  // the attribute is a property of the kernel: set it once per process
        if (!done) {
            cudaFuncSetAttribute(mm_adjoint2_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)MMTile<kF32>::kBytes);
            done = true;
        }
        mm_adjoint2_kernel<M><<<grid, kTileThreads, MMTile<kF32>::kBytes, st>>>(A1, A2, T);
    });
    return 1;
}

int mm_launch_adjoint_terminal(const AdjointArgs& A, int n_plane, cudaStream_t st) {
    with_media(A.a.media_mode, [&](auto mc) {
        constexpr int M = decltype(mc)::value;
        mm_adjoint_terminal_kernel<M><<<blocks_for(n_plane), kBlock, 0, st>>>(A, n_plane);
    });
    return 1;
}

int mm_fused2_occupancy(int storage, int media_mode) {
    int blocks = 0;
    with_pass_storage(storage, [&](auto sc) {
        with_media(media_mode, [&](auto mc) {
            constexpr int S = decltype(sc)::value, M = decltype(mc)::value;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, mm_fused2_kernel<S, M>, kFusedThreads, 0);
        });
    });
    return blocks;
}

int mm_launch_fused2(const StepArgs& aA, const StepArgs& aB, const FusedArgs& F, cudaStream_t st) {
    if (aA.storage == kF24) return 0;  // no 24-bit form of the passes
    const int grid = fused_grid(mm_fused2_occupancy(aA.storage, aA.media_mode));
    with_pass_storage(aA.storage, [&](auto sc) {
        with_media(aA.media_mode, [&](auto mc) {
            constexpr int S = decltype(sc)::value, M = decltype(mc)::value;
            mm_fused2_kernel<S, M><<<grid, kFusedThreads, 0, st>>>(aA, aB, F);
        });
    });
    return 1;
}

template <int S, int M, bool kRecord = false>
void mm_tile2_prepare() {
    static bool done = false;  // the attribute is a property of the kernel: set it once per process
    if (!done) {
        cudaFuncSetAttribute(mm_tile2_kernel<S, M, kRecord>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)MMTile<S>::kBytes);
        done = true;
    }
}

int mm_tile2_occupancy(int storage, int media_mode) {
    int blocks = 0;
    with_pass_storage(storage, [&](auto sc) {
        with_media(media_mode, [&](auto mc) {
            constexpr int S = decltype(sc)::value, M = decltype(mc)::value;
            mm_tile2_prepare<S, M>();
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, mm_tile2_kernel<S, M>, kTileThreads,
                                                          MMTile<S>::kBytes);
        });
    });
    return blocks;
}

int mm_launch_tile2(const StepArgs& aA, const StepArgs& aB, const TileArgs& T, cudaStream_t st) {
    if (aA.storage == kF24) return 0;  // no 24-bit form of the passes
    const dim3 grid(T.tiles_x * T.tiles_y, (aA.g.nz + T.chunk - 1) / T.chunk);
    with_pass_storage(aA.storage, [&](auto sc) {
        with_media(aA.media_mode, [&](auto mc) {
            constexpr int S = decltype(sc)::value, M = decltype(mc)::value;
            mm_tile2_prepare<S, M>();
            mm_tile2_kernel<S, M><<<grid, kTileThreads, MMTile<S>::kBytes, st>>>(aA, aB, T);
        });
    });
    return 1;
}

int mm_launch_record_tile2(const StepArgs& aA, const StepArgs& aB, const TileArgs& T, cudaStream_t st) {
    if (aA.storage != kF32 || !aA.rec || !aB.rec) return 0;
    const dim3 grid(T.tiles_x * T.tiles_y, (aA.g.nz + T.chunk - 1) / T.chunk);
    with_media(aA.media_mode, [&](auto mc) {
        constexpr int M = decltype(mc)::value;
        mm_tile2_prepare<kF32, M, true>();
        mm_tile2_kernel<kF32, M, true><<<grid, kTileThreads, MMTile<kF32>::kBytes, st>>>(aA, aB, T);
    });
    return 1;
}

int mm_halo_dirs(int vz_sign, int* dirs) {
    int k = 0;
    for (int d = 0; d < 12; ++d)
        if (kMMV[d][2] == vz_sign) dirs[k++] = d;
    return k;
}

int mm_launch_record_step(const StepArgs& a, cudaStream_t st) {
    int launched = 0;
    const bool rho = a.rho_in != nullptr;
    with_media(a.media_mode, [&](auto mc) {
        constexpr int M = decltype(mc)::value;
        if (rho) mm_record_kernel<M, true><<<blocks_for(a.g.n), kBlock, 0, st>>>(a);
        else mm_record_kernel<M, false><<<blocks_for(a.g.n), kBlock, 0, st>>>(a);
        launched = 1;
    });
    return launched;
}

}  // namespace lbm
