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

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace lbm {

constexpr int kMaxSources = 16;
constexpr int kBlock = 256;

enum MediaMode { kUniform = 0, kTable = 1, kPerCell = 2 };

// Population storage. Arithmetic is FP32 in every case; 16- and 24-bit storage convert at the pull
// and the store. A stored value is f * scale (scale a power of two, so the scaling itself is exact).
// kF24: an FP16 value h plus an 8-bit correction in units of ulp(h) / 256 (see F24 below).
enum StorageKind { kF32 = 0, kBF16 = 1, kF16 = 2, kF24 = 3 };

// Lattice shape. Cell coordinates come from the linear index by multiplication with host-computed
// magic numbers (Granlund and Montgomery, "Division by invariant integers using multiplication"):
// floor(i / d) = (i * M) >> (32 + k) with k = ceil(log2 d), M = ceil(2^(32+k) / d), exact for every
// i < 2^31.
struct Geometry {
    int nx, ny, nz;
    int n;  // nx * ny * nz, < 2^31
    unsigned long long mx, mxy;  // magic multipliers for division by nx and by nx * ny
    int kx, kxy;
};

// Per-material coefficients, computed on the host in double precision and rounded once (reciprocals
// as RN(1/d) of the stored float d, so that div_rn below is exact).
//   MM: c0 = (eps_r, 1/eps_r, g = 1/(1 + mu0 sigma/(4 eps_r)), 1/(4 mu_r)),  c1 = (sigma, mu_r, 0, 0)
//   HV: c0 = (eps, 1/eps, mu, 1/mu) with eps = eps0 eps_r, mu = mu0 mu_r,   c1 = (sigma, eps_r, 0, 0)
struct MatCoef {
    float4 c0, c1;
};

// Media as the kernels see them.
struct MediaView {
    MatCoef uniform;         // kUniform
    const uint8_t* id;       // kTable: material id per cell
    const MatCoef* table;    // kTable: coefficients per material
    const float* eps_r;      // kPerCell: raw values; coefficients are formed per cell
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
    const int* block_begin;       // [blocks + 1] for the blocks of kBlock cells of the step range
                                  // [cell_begin, cell_end): where each block's cells start in `cell`
                                  // (null without source cells)
};

// The source cells of block `b` of a launch over the step range (one thread per cell), recomputed
// after the block's ordinary updates: a barrier, so that their values replace the ordinary ones,
// then update(i, m) for every source cell i = cell[m] of the block. Every thread of the block must
// call this (the barrier), whether or not it had a cell of its own.
template <class Update>
__device__ __forceinline__ void block_source_cells(const SourceView& sv, int b, Update&& update) {
    if (!sv.block_begin) return;
    const int lo = sv.block_begin[b], hi = sv.block_begin[b + 1];
    if (hi <= lo) return;
    __syncthreads();
    for (int m = lo + (int)threadIdx.x; m < hi; m += (int)blockDim.x) update(sv.cell[m], m);
}

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
    int storage;      // StorageKind
    float scale;      // 16-bit storage: stored = f * scale
    float inv_scale;  // 1 / scale
    float* rec;       // adjoint record of this step (recording kernels only): kRecordFloats[model] x n
    int cell_begin, cell_end;  // cells the step and reduction launches cover (a z-slab skips its ghost planes)
};

// Per-cell record an adjoint step needs from its forward step: MM X = D' - mu0 J_ext / 4 (E is an
// exact function of X and the medium, recomputed by the same operations), HV E.
constexpr int kRecordFloatsMM = 3;
constexpr int kRecordFloatsHV = 3;

// Field output: for each selected field a 3 x n block; null pointers are skipped.
struct FieldsOut {
    float* E;
    float* B;
    float* D;
    float* H;
    float* J;
};

// --- population storage traits -----------------------------------------------------------
// Pack4<S>: four populations (one MM direction group, or HV's e_x, e_y, e_z, h_x) as one vector;
// Pack2<S>: two populations (HV's h_y, h_z). FP32: float4 / float2; 16-bit: 8 / 4 bytes.
template <int S>
struct Pack4;
template <int S>
struct Pack2;

template <>
struct Pack4<kF32> {
    using T = float4;
    __device__ static float4 unpack(T u, float) { return u; }
    __device__ static float4 load(const T* p, float) { return __ldg(p); }
    __device__ static T pack(float4 v, float) { return v; }
};
template <>
struct Pack2<kF32> {
    using T = float2;
    __device__ static float2 unpack(T u, float) { return u; }
    __device__ static float2 load(const T* p, float) { return __ldg(p); }
    __device__ static T pack(float2 v, float) { return v; }
};

template <>
struct Pack4<kF16> {
    using T = uint2;
    __device__ static float4 load(const T* p, float inv) { return unpack(__ldg(p), inv); }
    __device__ static float4 unpack(T u, float inv) {
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
        return make_float4(a.x * inv, a.y * inv, b.x * inv, b.y * inv);
    }
    __device__ static T pack(float4 v, float scale) {
        const __half2 a = __floats2half2_rn(v.x * scale, v.y * scale);
        const __half2 b = __floats2half2_rn(v.z * scale, v.w * scale);
        return make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
    }
};
template <>
struct Pack2<kF16> {
    using T = uint32_t;
    __device__ static float2 load(const T* p, float inv) { return unpack(__ldg(p), inv); }
    __device__ static float2 unpack(T u, float inv) {
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u));
        return make_float2(a.x * inv, a.y * inv);
    }
    __device__ static T pack(float2 v, float scale) {
        const __half2 a = __floats2half2_rn(v.x * scale, v.y * scale);
        return *reinterpret_cast<const uint32_t*>(&a);
    }
};

template <>
struct Pack4<kBF16> {
    using T = uint2;
    __device__ static float4 load(const T* p, float inv) { return unpack(__ldg(p), inv); }
    __device__ static float4 unpack(T u, float inv) {
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
        return make_float4(a.x * inv, a.y * inv, b.x * inv, b.y * inv);
    }
    __device__ static T pack(float4 v, float scale) {
        const __nv_bfloat162 a = __floats2bfloat162_rn(v.x * scale, v.y * scale);
        const __nv_bfloat162 b = __floats2bfloat162_rn(v.z * scale, v.w * scale);
        return make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
    }
};
template <>
struct Pack2<kBF16> {
    using T = uint32_t;
    __device__ static float2 load(const T* p, float inv) { return unpack(__ldg(p), inv); }
    __device__ static float2 unpack(T u, float inv) {
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
        return make_float2(a.x * inv, a.y * inv);
    }
    __device__ static T pack(float2 v, float scale) {
        const __nv_bfloat162 a = __floats2bfloat162_rn(v.x * scale, v.y * scale);
        return *reinterpret_cast<const uint32_t*>(&a);
    }
};

// 24-bit storage. A value x (already scaled) is kept as h = x rounded toward zero to FP16 and an
// unsigned byte q = |x - h| / (ulp(h) / 256) rounded to nearest, where ulp(h) = 2^(max(E, 1) - 25)
// for h's biased exponent E (2^-24 for zero and subnormal h). x - h is exact in FP32 (h is x cut to
// fewer digits) and lies in [0, ulp(h)) in magnitude, so q is 0 ... 256; 256 carries into h, which
// moves one FP16 value away from zero (the bit pattern + 1), with q = 0, exactly. The value
// h + sign(h) q ulp(h) / 256 then keeps 19 significant bits where FP16 keeps 11 (relative error at
// most 2^-19 for normal h), and it decodes exactly: it needs at most 20 bits. |x| beyond FP16's
// largest value saturates there. The halves of a direction group and their bytes live in separate
// planes (a group's 4 halves as one 8-byte word, its 4 bytes as one 4-byte word), so each is one
// coalesced access.
//
// The common cases are computed without branches and without conversion instructions, on the
// value's FP32 bits. Write W for the FP32 pattern of |stored value| * 2^-112: for a normal h it is
// [0][e5 as the exponent field][h's 10 mantissa bits][q][5 zero bits], for a zero or subnormal h the
// denormal (h's bits * 256 + q) * 2^5; in both cases W = (h without its sign) << 13 | q << 5.
//   Decode: W from the stored bits, then W * 2^112 * 2^112, the sign, * 2^-112 / scale. The first
//   product is exact; the second overflows to infinity exactly for h's infinities and NaN (exponent
//   31, values >= 2^16; a NaN decodes as an infinity), and is exact otherwise. Denormal W needs FP32
//   denormals kept, which this build does (no flush to zero).
//   Encode, 2^-14 <= |x| < 2^15 (h normal): |x| * 2^-112 is exact and normal; its bits rounded to
//   nearest at bit 5 (halves to even) are W. |x| < 2^-14: |x| + 2^-9 rounds |x| to a multiple of
//   2^-32 (halves to even) and its low 23 bits are h's bits * 256 + q. Either way a carry out of q
//   runs into h, as the definition's carry does.
//   |x| >= 2^15, infinities and NaN go to encode_rare, the definition written out.
static __device__ __noinline__ void f24_encode_rare(float x, unsigned& h, unsigned& q);
struct F24 {
    __device__ static float join(unsigned z, float inv) {  // z: h in bits 31..16, q in bits 15..8
        const float w = __uint_as_float((z >> 3) & 0x0fffffe0u);
        const float m = (w * 0x1p112f) * 0x1p112f;
        return (__uint_as_float(__float_as_uint(m) | (z & 0x80000000u)) * 0x1p-112f) * inv;
    }
    // Bits of the stored pair of x = v * scale: h in bits 15..0, q in bits 23..16 (for packing).
    __device__ static unsigned split(float v, float scale) {
        const float x = v * scale, a = fabsf(x);
        const unsigned b = __float_as_uint(x);
        const unsigned zn = __float_as_uint(a * 0x1p-112f);
        const unsigned wn = zn + 0xfu + ((zn >> 5) & 1u);                         // to nearest at bit 5
        const unsigned ws = (__float_as_uint(a + 0x1p-9f) & 0x7fffffu) << 5;       // multiple of 2^-32
        const unsigned w = (a < 0x1p-14f ? ws : wn) | ((b >> 3) & 0x10000000u);    // sign into bit 28
        unsigned out = (w >> 13) | ((w << 11) & 0x00ff0000u);
        if (!(a < 0x1p15f)) {
            unsigned h, q;
            f24_encode_rare(x, h, q);
            out = h | (q << 16);
        }
        return out;
    }
    // Four values: halves at hi[idx], bytes at lo[idx].
    __device__ static float4 load4(const uint2* hi, const unsigned* lo, size_t idx, float inv) {
        const uint2 h = __ldg(hi + idx);
        const unsigned q = __ldg(lo + idx);
        return make_float4(join(__byte_perm(h.x, q, 0x1040), inv), join(__byte_perm(h.x, q, 0x3250), inv),
                           join(__byte_perm(h.y, q, 0x1060), inv), join(__byte_perm(h.y, q, 0x3270), inv));
    }
    __device__ static void store4(uint2* hi, unsigned* lo, size_t idx, float4 v, float scale) {
        const unsigned s0 = split(v.x, scale), s1 = split(v.y, scale), s2 = split(v.z, scale), s3 = split(v.w, scale);
        hi[idx] = make_uint2(__byte_perm(s0, s1, 0x5410), __byte_perm(s2, s3, 0x5410));
        lo[idx] = __byte_perm(__byte_perm(s0, s1, 0x0062), __byte_perm(s2, s3, 0x0062), 0x5410);
    }
    // Two values: halves at hi[idx], bytes at lo[idx].
    __device__ static float2 load2(const unsigned* hi, const unsigned short* lo, size_t idx, float inv) {
        const unsigned h = __ldg(hi + idx);
        const unsigned q = __ldg(lo + idx);
        return make_float2(join(__byte_perm(h, q, 0x1040), inv), join(__byte_perm(h, q, 0x3250), inv));
    }
    __device__ static void store2(unsigned* hi, unsigned short* lo, size_t idx, float2 v, float scale) {
        const unsigned s0 = split(v.x, scale), s1 = split(v.y, scale);
        hi[idx] = __byte_perm(s0, s1, 0x5410);
        lo[idx] = (unsigned short)__byte_perm(s0, s1, 0x0062);
    }
};

// The definition itself, for |x| >= 2^15, infinities and NaN (x already scaled).
static __device__ __noinline__ void f24_encode_rare(float x, unsigned& h, unsigned& q) {
    const __half hh = __float2half_rz(x);
    h = __half_as_ushort(hh);
    const float r = fabsf(x - __half2float(hh));
    const unsigned e = max((h >> 10) & 0x1fu, 1u);
    const int k = __float2int_rn(r * __uint_as_float((160u - e) << 23));  // |r| / 2^(e - 33)
    if (k < 256) {
        q = (unsigned)max(k, 0);
    } else if (k == 256 && (h & 0x7fffu) < 0x7bffu) {
        h += 1;  // the next FP16 value away from zero
        q = 0;
    } else {
        q = 255;  // beyond FP16's largest value
    }
}

// Host-side dispatch of a runtime storage kind / media mode to a compile-time constant.
template <class F>
inline void with_storage(int s, F&& f) {
    if (s == kBF16) f(std::integral_constant<int, kBF16>{});
    else if (s == kF16) f(std::integral_constant<int, kF16>{});
    else if (s == kF24) f(std::integral_constant<int, kF24>{});
    else f(std::integral_constant<int, kF32>{});
}
// The same for the two-step passes, which keep populations in their storage format in shared
// memory or L2 and have no 24-bit form (the host never selects a pass for kF24 storage).
template <class F>
inline void with_pass_storage(int s, F&& f) {
    if (s == kBF16) f(std::integral_constant<int, kBF16>{});
    else if (s == kF16) f(std::integral_constant<int, kF16>{});
    else if (s == kF32) f(std::integral_constant<int, kF32>{});
}
template <class F>
inline void with_media(int m, F&& f) {
    if (m == kTable) f(std::integral_constant<int, kTable>{});
    else if (m == kPerCell) f(std::integral_constant<int, kPerCell>{});
    else f(std::integral_constant<int, kUniform>{});
}

inline int blocks_for(int n) { return (n + kBlock - 1) / kBlock; }

// Grid of a persistent launch: resident blocks per SM x the current device's SM count.
inline int fused_grid(int blocks_per_sm) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return std::max(1, blocks_per_sm) * std::max(1, sms);
}

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
    int x, y, z;
};

__device__ __forceinline__ Neighbourhood neighbourhood(const Geometry& g, int i) {
    const int nxy = g.nx * g.ny;
    const int z = (int)(((unsigned long long)(unsigned)i * g.mxy) >> (32 + g.kxy));
    const int r = i - z * nxy;
    const int y = (int)(((unsigned long long)(unsigned)r * g.mx) >> (32 + g.kx));
    const int x = r - y * g.nx;
    Neighbourhood h;
    h.x = x;
    h.y = y;
    h.z = z;
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

// Ask L2 to fetch the line holding p ahead of a load of it; nothing waits for it and no register
// receives it. Callers pass only addresses they are about to load themselves.
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Prefetch into L2 the medium of cell i (nothing for a uniform medium).
template <int M>
__device__ __forceinline__ void prefetch_media(const MediaView& m, int i) {
    if constexpr (M == kTable) {
        prefetch_l2(&m.id[i]);
    } else if constexpr (M == kPerCell) {
        prefetch_l2(&m.eps_r[i]);
        prefetch_l2(&m.mu_r[i]);
        prefetch_l2(&m.sigma[i]);
    }
}

// Index of the cell at offset (sx, sy, sz) in {-1, 0, 1}^3.
template <int SX, int SY, int SZ>
__device__ __forceinline__ int shifted(const Neighbourhood& h) {
    return h.xo[SX + 1] + h.yo[SY + 1] + h.zo[SZ + 1];
}

// x / d rounded to nearest, from r = RN(1/d): q = RN(x r), e = x - q d (exact with a fused
// multiply-add), result RN(q + e r). By Markstein's theorem on FMA-based division this is the
// correctly rounded quotient (away from underflow and overflow), without a divide instruction or
// its special-case branch.
__device__ __forceinline__ float div_rn(float x, float d, float r) {
    const float q = __fmul_rn(x, r);
    const float e = __fmaf_rn(-q, d, x);
    return __fmaf_rn(e, r, q);
}

enum ModelKind { kModelMM = 0, kModelHV = 1 };

// Coefficients of cell i. Per-cell media form them here from the raw values (true divisions).
template <int Model, int M>
__device__ __forceinline__ MatCoef load_coef(const MediaView& m, int i, float eps0, float mu0) {
    if constexpr (M == kUniform) {
        return m.uniform;
    } else if constexpr (M == kTable) {
        const MatCoef* t = &m.table[__ldg(&m.id[i])];
        MatCoef c;
        c.c0 = __ldg(&t->c0);
        c.c1 = __ldg(&t->c1);
        return c;
    } else {
        const float er = __ldg(&m.eps_r[i]), mr = __ldg(&m.mu_r[i]), sg = __ldg(&m.sigma[i]);
        MatCoef c;
        if constexpr (Model == kModelMM) {
            c.c0 = make_float4(er, 1.f / er, 1.f / (1.f + 0.5f * (sg / er)), 0.25f / mr);
            c.c1 = make_float4(sg, mr, 0.f, 0.f);
        } else {
            const float eps = eps0 * er, mu = mu0 * mr;
            c.c0 = make_float4(eps, 1.f / eps, mu, 1.f / mu);
            c.c1 = make_float4(sg, er, 0.f, 0.f);
        }
        return c;
    }
}

// External current and imposed fields of special cell m at the current step.
struct CellSource {
    float3 J;
    float3 E;
    float3 B;
    bool imposed;
};

// The sums are explicit fused multiply-adds, so that every kernel that inlines this gets the same bits.
__device__ __forceinline__ CellSource cell_source(const SourceView& sv, const SourceScalars& sc, int m) {
    CellSource cs;
    cs.J = make_float3(0.f, 0.f, 0.f);
    cs.E = make_float3(0.f, 0.f, 0.f);
    cs.B = make_float3(0.f, 0.f, 0.f);
    const int b = sv.entry_begin[m], e = sv.entry_begin[m + 1];
    for (int k = b; k < e; ++k) {
        const float s = sc.s[sv.entry_src[k]];
        cs.J.x = __fmaf_rn(sv.entry_w[3 * k + 0], s, cs.J.x);
        cs.J.y = __fmaf_rn(sv.entry_w[3 * k + 1], s, cs.J.y);
        cs.J.z = __fmaf_rn(sv.entry_w[3 * k + 2], s, cs.J.z);
    }
    const uint32_t mask = sv.impose_mask[m];
    cs.imposed = mask != 0u;
    for (int k = 0; k < kMaxSources; ++k) {
        if ((mask >> k) & 1u) {
            const float s = sc.s[k];
            cs.E.x = __fmaf_rn(sc.E0[k][0], s, cs.E.x);
            cs.E.y = __fmaf_rn(sc.E0[k][1], s, cs.E.y);
            cs.E.z = __fmaf_rn(sc.E0[k][2], s, cs.E.z);
            cs.B.x = __fmaf_rn(sc.B0[k][0], s, cs.B.x);
            cs.B.y = __fmaf_rn(sc.B0[k][1], s, cs.B.y);
            cs.B.z = __fmaf_rn(sc.B0[k][2], s, cs.B.z);
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

// --- batched stepping of several lattices -------------------------------------------------
// One lattice of a batch as the batched kernels read it from device memory. The host rewrites the
// array before every batched call, so a captured graph of the call replays on fresh contents.
struct BatchLattice {
    StepArgs base;         // geometry, media, special cells, imposed vectors, storage, eps0, mu0
    void* buf[2];          // population buffers; step j reads buf[(cur0 + j) & 1]
    void* buf2[2];         // HV second arrays (MM: unused)
    float* rho[2];         // MM rest population f_0^(0) when tracked, else null
    const float* s_table;  // source values s_k(t0 + j + 1) at [k * s_stride + j]
    int s_stride;
    int n_src;
    int cur0;   // buffer index holding the state when the call starts
    int steps;  // steps this lattice advances in the call
};

// A block's share of the batch: cells [begin, begin + blockDim) of one lattice (or, for the
// source-cell launch, special cells [begin, begin + blockDim)).
struct BatchTile {
    int lattice;
    int begin;
};

// StepArgs of lattice L at batch step j (buffers and storage; sources are filled by the caller).
__device__ __forceinline__ StepArgs batch_args(const BatchLattice* __restrict__ L, int j) {
    StepArgs a;
    a.g = L->base.g;
    a.media_mode = L->base.media_mode;
    a.media = L->base.media;
    const int in = (L->cur0 + j) & 1, out = in ^ 1;
    a.fin = L->buf[in];
    a.fout = L->buf[out];
    a.fin2 = L->buf2[in];
    a.fout2 = L->buf2[out];
    a.rho_in = L->rho[in];
    a.rho_out = L->rho[out];
    a.eps0 = L->base.eps0;
    a.mu0 = L->base.mu0;
    a.storage = L->base.storage;
    a.scale = L->base.scale;
    a.inv_scale = L->base.inv_scale;
    a.sv = L->base.sv;
    return a;
}

// Source values of lattice L at batch step j, and its imposed-field vectors.
__device__ __forceinline__ void batch_sources(const BatchLattice* __restrict__ L, int j, StepArgs& a) {
    for (int k = 0; k < L->n_src; ++k) {
        a.sc.s[k] = L->s_table[k * L->s_stride + j];
        for (int q = 0; q < 3; ++q) {
            a.sc.E0[k][q] = L->base.sc.E0[k][q];
            a.sc.B0[k][q] = L->base.sc.B0[k][q];
        }
    }
}

struct BatchLaunch {
    const BatchLattice* lat;
    const BatchTile* tiles;   // main tiles, lattices in decreasing step count
    const BatchTile* stiles;  // special-cell tiles, same lattice order
    int block;                // threads per block of the main launch (128 or 256)
    int grid_cap;             // persistent launch: blocks in the grid (0 = one block per tile)
    int storage;
    bool rho;
};

// --- adjoint (gradients of a plane loss with respect to eps_r and sigma) ---------------------
// One backward step reverses the forward iteration n -> n+1. nu^{n+1} = dL/df^{n+1} holds the adjoint
// of every cell's pre-collision populations (FP32, the population group layout). The adjoint of
// cell x's post-collision values is nu^{n+1} at x + v_d (advection reversed); the transposed
// collision gives nu^n(x), plus the derivative of the loss of time n when x lies in the loss plane.
struct AdjointArgs {
    StepArgs a;            // media, sources of iteration n + 1; record of the forward step in a.rec
                           // (the terminal launch reads the final state from a.fin / a.fin2 instead)
    const void* nu_in;     // nu^{n+1} (null for the terminal launch)
    const void* nu_in2;    // HV second array
    void* nu_out;          // nu^n
    void* nu_out2;
    float* grad_eps;       // dL/d eps_r per cell, accumulated
    float* grad_sigma;     // dL/d sigma per cell, accumulated (null: not computed)
    const uint8_t* special_mask;  // non-zero at source cells, which the second launch handles
    int plane_axis, plane_index;  // loss plane: cells whose coordinate on plane_axis is plane_index
    int loss_active;              // add the plane loss term of time n
    double* loss_plane;           // |E|^2 summed over time, per plane cell (slot k as in plane_cell);
                                  // the terminal launch writes it, the others add
};

// Cells of the loss plane, and whether a cell lies in it.
__device__ __forceinline__ int plane_cells(const Geometry& g, int axis) {
    return axis == 0 ? g.ny * g.nz : (axis == 1 ? g.nx * g.nz : g.nx * g.ny);
}
__device__ __forceinline__ int plane_cell(const Geometry& g, int axis, int index, int k) {
    if (axis == 0) return index + g.nx * k;  // k = y + ny z
    if (axis == 1) {
        const int z = k / g.nx, x = k - z * g.nx;
        return x + g.nx * (index + g.ny * z);
    }
    return k + g.nx * g.ny * index;  // k = x + nx y
}
// Slot k of a plane cell: the inverse of plane_cell.
__device__ __forceinline__ int plane_slot(const Neighbourhood& h, const Geometry& g, int axis) {
    return axis == 0 ? h.y + g.ny * h.z : (axis == 1 ? h.x + g.nx * h.z : h.x + g.nx * h.y);
}
__device__ __forceinline__ bool in_plane(const Neighbourhood& h, const Geometry& g, int axis, int index) {
    if (axis == 0) return h.xo[1] == index;
    if (axis == 1) return h.yo[1] == index * g.nx;
    return h.zo[1] == index * g.nx * g.ny;
}

// |E|^2 of a plane cell into its loss slot: written by the terminal launch (time T), then added by
// the launch of each earlier time, so every slot sums its times in the order T, T-1, ..., 1.
template <bool kFirst>
__device__ __forceinline__ void add_plane_loss(const AdjointArgs& A, const Neighbourhood& h, float3 E) {
    const double e2 = (double)E.x * E.x + (double)E.y * E.y + (double)E.z * E.z;
    double* slot = A.loss_plane + plane_slot(h, A.a.g, A.plane_axis);
    if constexpr (kFirst) *slot = e2;
    else *slot += e2;
}

// --- two time steps per pass over the populations ---------------------------------------------
// A step of cell x reads only the populations of its 3 x 3 x 3 neighbourhood. So step t + 1 of a
// cell can run as soon as step t has produced its 27 neighbours. One persistent launch runs both
// steps as a wavefront along z:
//   phase A(p): step t of plane p, from the A/B buffer into an intermediate plane;
//   phase B(p): step t + 1 of plane p, from the intermediate planes p - 1, p, p + 1 into the other
//     A/B buffer.
// The intermediate planes of 1 .. nz - 2 live in a ring of R plane slots, small enough to stay in
// L2. Planes 0 and nz - 1 are needed at both ends of the periodic wavefront, so they have slots
// of their own. Each step's HBM traffic is then one read or one write of the populations instead
// of both.
// Phases run in the order A(nz-1), A(0), .., A(L-1), then B(k), A(k + L) for k = 0 .. nz-2-L,
// then the remaining B phases (L >= 2: B(k) needs A(k + 1); R >= L + 1 keeps every wait on an
// earlier item). A phase is `tiles` tiles of tile_cells consecutive cells of its plane. A tile
// also recomputes the source cells among its own cells (after a barrier of its compute threads, so
// that their values replace those of the ordinary update), so a finished tile is final, however
// many source cells a plane holds. Blocks take tiles in that order from a counter, and a tile waits
// only for tiles taken before it:
//   * tile j of B(p) waits for the tiles of A(p - 1), A(p), A(p + 1) holding the rows next to its
//     own (the cells it pulls from);
//   * tile j of A(p) waits for the same neighbourhood of tiles of the three B phases that read the
//     slot's previous plane, p - R.
// Tiles publish the pass number in a flag of their own, so the flags need no reset between passes.
// Every wait has a time limit; past it the pass sets `abort` and every block stops. A negative
// limit makes every item that depends on another give up at its first check, met or not: the host
// uses it to drive the time-out path deterministically in tests.
struct FusedArgs {
    void* ring;   // R slots of one plane of intermediate populations (the model's group layout)
    void* lo;     // slot of plane 0
    void* hi;     // slot of plane nz - 1
    void* ring2;  // HV: the same for the pair arrays (null for MM)
    void* lo2;
    void* hi2;
    int R;
    int L;                      // A runs L planes ahead of B in the item order (R >= L + 1)
    int tile_cells;             // cells per tile: a multiple of kBlock (each thread takes every kBlock-th)
    int tiles;                  // tiles per plane
    int epoch;                  // this pass's number (>= 1); flags hold the last pass they finished
    int* next;                  // item counter (zero at launch)
    int* tile_flag;             // 2 nz tiles flags, A then B
    int* abort;                 // set when a wait timed out
    const int* tile_special;    // nz tiles + 1 offsets of each tile's cells in the special-cell list
    long long timeout_ns;       // < 0: give up at the first dependency check
};

enum { kPhaseA = 0, kPhaseB = 1 };

__host__ __device__ __forceinline__ void fused_phase(int q, int nz, int L, int* type, int* plane) {
    if (q < L + 1) {
        *type = kPhaseA;
        *plane = q == 0 ? nz - 1 : q - 1;
        return;
    }
    const int j = q - (L + 1), pairs = nz - 1 - L;
    if (j < 2 * pairs) {
        *type = (j & 1) ? kPhaseA : kPhaseB;
        *plane = (j & 1) ? (j >> 1) + L : (j >> 1);
        return;
    }
    *type = kPhaseB;
    *plane = pairs + (j - 2 * pairs);
}

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int load_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait until *ctr >= target; false when the pass was aborted or the wait timed out (then aborts).
// The loop does not sleep: the L2 round trip of each look paces it, and the pass is bound by how
// soon a published item is seen (sleeping backoff measured 0.6 % (MM) and 1 % (HV) slower).
__device__ inline bool fused_wait(const FusedArgs& F, const int* ctr, int target) {
    if (load_acquire(ctr) >= target) return true;
    const long long t0 = global_ns();
    while (load_acquire(ctr) < target) {
        if (load_acquire(F.abort)) return false;
        if (global_ns() - t0 > F.timeout_ns) {
            atomicExch(F.abort, 1);
            return false;
        }
    }
    return true;
}

// Tiles holding the rows y0 - 1 .. y1 + 1 (cyclically) around the rows y0 .. y1 of tile j: the
// first tile and how many. A cell pulls from (x +- 1, y +- 1), and the x wrap stays in its row.
__host__ __device__ __forceinline__ void tile_window(int j, int tiles, int tile_cells, int nx, int nxy, int* first,
                                                     int* count) {
    const int c0 = j * tile_cells, c1 = (c0 + tile_cells < nxy ? c0 + tile_cells : nxy) - 1;
    const int y0 = c0 / nx, y1 = c1 / nx;
    const long long span = (long long)(y1 - y0 + 3) * nx;
    if (span >= nxy) {
        *first = 0;
        *count = tiles;
        return;
    }
    int lo = (y0 - 1) * nx;
    if (lo < 0) lo += nxy;
    const int hi = lo + (int)span - 1;  // may pass nxy: wraps
    *first = lo / tile_cells;
    *count = hi < nxy ? hi / tile_cells - *first + 1 : (tiles - *first) + ((hi - nxy) / tile_cells + 1);
    if (*count > tiles) *count = tiles;
}

// The phases a tile of phase (type, plane) waits for: the tiles of planes q[0..2] in phase *wtype
// within its window. B(p) reads the intermediate planes p - 1, p, p + 1 written by A; A(p) rewrites
// the ring slot whose previous plane, p - R, the B phases p - R - 1 .. p - R + 1 read. Returns the
// number of planes (0: nothing to wait for).
__host__ __device__ __forceinline__ int fused_waits_on(int type, int plane, int nz, int R, int* wtype, int* q) {
    if (type == kPhaseB) {
        *wtype = kPhaseA;
        q[0] = (plane + nz - 1) % nz;
        q[1] = plane;
        q[2] = (plane + 1) % nz;
        return 3;
    }
    const int prev = plane - R;
    if (!(plane >= 1 && plane <= nz - 2 && prev >= 1)) return 0;
    *wtype = kPhaseB;
    q[0] = prev - 1;
    q[1] = prev;
    q[2] = prev + 1;
    return 3;
}

// An item of a pass: tile j of phase (type, plane).
struct FusedItem {
    int type, plane, j;
};

__device__ __forceinline__ FusedItem fused_item(int item, int tiles, int nz, int L) {
    FusedItem it;
    const int q = item / tiles;
    it.j = item - q * tiles;
    fused_phase(q, nz, L, &it.type, &it.plane);
    return it;
}

// Dependencies of item `it`, checked by the 32 lanes of one warp at once: the tile flags of three
// planes' windows are spread over the lanes, so a satisfied item costs one round of loads. `own`
// is the item the same block runs just before this one: it is complete by the time this one
// starts (the block's barriers order it), so it is not waited for. Same verdict in every lane.
__device__ inline bool fused_ready_warp(const FusedArgs& F, int nz, FusedItem it, FusedItem own, int nx, int nxy,
                                        bool wait) {
    const int lane = threadIdx.x & 31;
    bool ok = true;
    // one look (wait == false) or a bounded wait
    auto reached = [&](const int* p, int target) { return wait ? fused_wait(F, p, target) : load_acquire(p) >= target; };
    int q[3];
    int wtype = 0;
    if (fused_waits_on(it.type, it.plane, nz, F.R, &wtype, q) == 0) return true;
    if (F.timeout_ns < 0) {  // negative limit: stop the pass at the first item with a dependency
        if (lane == 0) atomicExch(F.abort, 1);
        return false;
    }
    int first, count;
    tile_window(it.j, F.tiles, F.tile_cells, nx, nxy, &first, &count);
    for (int idx = lane; ok && idx < 3 * count; idx += 32) {
        const int k = idx / count;
        int t = first + (idx - k * count);
        if (t >= F.tiles) t -= F.tiles;
        if (own.type == wtype && own.plane == q[k] && own.j == t) continue;
        ok = reached(F.tile_flag + ((size_t)wtype * nz + q[k]) * F.tiles + t, F.epoch);
    }
    return __all_sync(0xffffffffu, ok);
}

// Publish a finished tile (after every store of the block: the caller's barrier orders them).
__device__ __forceinline__ void fused_publish(const FusedArgs& F, int nz, FusedItem it) {
    __threadfence();
    atomicExch(F.tile_flag + ((size_t)it.type * nz + it.plane) * F.tiles + it.j, F.epoch);
}

// Threads of a two-step block: kBlock compute threads and one scheduler warp.
constexpr int kFusedThreads = kBlock + 32;

// Shared-memory slots of one compute thread of a two-step pass, a float2 each, laid out [slot]
// [compute thread] so that a warp's accesses do not conflict. Populations wait there between a
// cell's pull and its collision instead of holding registers: at the pass's 72 registers per
// thread the compiler would otherwise spill more to local memory, whose stores go through to L2
// (256^3 dipole on GB300: the MM pass 2.5 % and the HV pass 1.7 % faster with the slots). The
// accesses are volatile so that the compiler keeps the round trip instead of forwarding the
// stored values in registers.
struct FusedStash {
    static constexpr bool kStash = true;
    __device__ bool keeps_record() const { return true; }  // a recording step writes this cell's record
    unsigned slot;  // shared address of this thread's slot 0; slot k lies k * kBlock * 8 bytes on
    __device__ void stash_put(int k, float x, float y) const {
        asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(slot + k * kBlock * 8), "f"(x), "f"(y));
    }
    __device__ void stash_get(int k, float& x, float& y) const {
        asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(x), "=f"(y) : "r"(slot + k * kBlock * 8));
    }
};
// The same hooks for the single-step paths, which keep every value in registers.
struct NoStash {
    static constexpr bool kStash = false;
    __device__ bool keeps_record() const { return true; }  // a recording step writes this cell's record
    __device__ void stash_put(int, float, float) const {}
    __device__ void stash_get(int, float&, float&) const {}
};
__device__ __forceinline__ unsigned fused_stash_slot(const float2* slots) {
    return static_cast<unsigned>(__cvta_generic_to_shared(slots + threadIdx.x));
}

__device__ __forceinline__ void named_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// The persistent loop. The scheduler warp (threads kBlock ..) takes the next item from the
// counter and looks at its inputs while the kBlock compute threads run the current one:
//   compute: bar.sync(handoff) -> read the item -> work -> bar.arrive(done) -> repeat;
//   scheduler: take item n+1 and look once at its inputs -> bar.sync(done) (item n finished) ->
//     if they were all there: hand n+1 over (bar.arrive(handoff)), then publish n while it runs;
//     otherwise: publish n first, then wait for n+1's inputs and hand it over.
// Publishing never waits behind another item's inputs, so the earliest unpublished item can
// always proceed (every item waits only for earlier ones); and in the usual case neither the
// check nor the publication's fence delays the compute threads. Item n+1's dependence on n
// itself is not looked up: the block's barriers order n before n+1.
// The scheduler also works out what the compute threads need of an item (`describe`: phase,
// plane, tile and the ring slots it reads or writes) while they run the previous one, and hands
// it over in shared memory, so the compute threads do no index arithmetic per item.
struct FusedDesc {
    int type, plane, j;
    int s_lo, s_hi;  // the tile's source cells: entries s_lo .. s_hi - 1 of the special-cell list
    void* ptr[6];
};

// Barrier of a two-step block's compute threads alone (ids 1 and 2 are the hand-off barriers).
constexpr int kComputeBarrier = 3;

template <class Describe, class Work>
__device__ inline void fused_loop(const FusedArgs& F, int nx, int nxy, int nz, Describe&& describe, Work&& work) {
    constexpr int kHandoff = 1, kDone = 2;
    __shared__ int s_item[2], s_ok[2];
    __shared__ FusedDesc s_desc[2];
    const int per_phase = F.tiles;
    const int total = 2 * nz * per_phase;
    if (threadIdx.x < kBlock) {
        for (int buf = 0;; buf ^= 1) {
            named_sync(kHandoff, kFusedThreads);
            const int item = s_item[buf];
            if (item >= total || !s_ok[buf]) return;
            work(s_desc[buf]);
            named_arrive(kDone, kFusedThreads);
        }
    }
    // scheduler warp
    const int lane = threadIdx.x & 31;
    const FusedItem none{-1, -1, -1};
    auto make_desc = [&](const FusedItem& it) {
        FusedDesc d;
        d.type = it.type;
        d.plane = it.plane;
        d.j = it.j;
        const int* ts = F.tile_special + (size_t)it.plane * F.tiles + it.j;
        d.s_lo = ts[0];
        d.s_hi = ts[1];
        describe(it, d);
        return d;
    };
    int item = 0;
    if (lane == 0) item = atomicAdd(F.next, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    bool ok = item >= total || fused_ready_warp(F, nz, fused_item(item, per_phase, nz, F.L), none, nx, nxy, true);
    if (lane == 0) {
        s_item[0] = item;
        s_ok[0] = ok ? 1 : 0;
        if (item < total) s_desc[0] = make_desc(fused_item(item, per_phase, nz, F.L));
    }
    named_arrive(kHandoff, kFusedThreads);
    for (int buf = 1;; buf ^= 1) {
        if (item >= total || !ok) return;
        const FusedItem cur = fused_item(item, per_phase, nz, F.L);
        int nxt = 0;
        if (lane == 0) nxt = atomicAdd(F.next, 1);
        nxt = __shfl_sync(0xffffffffu, nxt, 0);
        const FusedItem next = nxt < total ? fused_item(nxt, per_phase, nz, F.L) : none;
        const bool ready = nxt >= total || fused_ready_warp(F, nz, next, cur, nx, nxy, false);
        if (lane == 0) {  // slot `buf` held the item before `cur`, which every compute thread has finished
            s_item[buf] = nxt;
            if (nxt < total) s_desc[buf] = make_desc(next);
        }
        named_sync(kDone, kFusedThreads);  // the compute threads finished `cur`
        bool ok2 = true;
        if (ready) {
            if (lane == 0) s_ok[buf] = 1;
            named_arrive(kHandoff, kFusedThreads);
            if (lane == 0) fused_publish(F, nz, cur);
        } else {
            if (lane == 0) fused_publish(F, nz, cur);
            __syncwarp();
            ok2 = fused_ready_warp(F, nz, next, none, nx, nxy, true);
            if (lane == 0) s_ok[buf] = ok2 ? 1 : 0;
            named_arrive(kHandoff, kFusedThreads);
        }
        item = nxt;
        ok = ok2;
    }
}

// --- two time steps per pass in shared memory (overlapped tiles) ------------------------------
// A block owns a tile of kTileTX x kTileTY cells of each plane of a chunk of planes, and one thread
// per cell of the tile and of a ring of one cell around it: kTileEX x kTileEY = (TX + 2) x (TY + 2)
// "extended" cells. Marching up its chunk, it steps plane p of the extended tile (phase A, step t:
// pulls from the A/B buffer in HBM, results into shared memory), then plane p - 1 of the tile
// itself (phase B, step t + 1: pulls from the shared planes p - 2, p - 1, p, results into the other
// A/B buffer). The ring is what phase B's pulls reach outside the tile, so blocks never wait for
// one another; the ring's cells are stepped twice (by this block and by their own), the price of
// that independence. The intermediate step never leaves the SM: each pair of steps reads and writes
// the populations in HBM once, and writes them into L2 only twice (the fill and the output).
// Phase B pulls a direction with v_z = +1 from plane p - 2, v_z = 0 from p - 1, v_z = -1 from p, so
// shared memory keeps each plane's directions by v_z class only as long as they are read: the
// v_z = -1 class of the newest plane, the v_z = 0 class of the last two and the v_z = +1 class of
// the last three. A tile recomputes the source cells of its extended cells after its ordinary
// update (after a barrier, so that their values replace the ordinary ones). The arithmetic is the
// single step's, so a pass equals two single steps bit for bit.
constexpr int kTileEX = 16, kTileEY = 16;  // extended tile: one thread per cell
constexpr int kTileTX = kTileEX - 2, kTileTY = kTileEY - 2;
constexpr int kTileThreads = kTileEX * kTileEY;

struct TileArgs {
    int tiles_x, tiles_y;  // tiles per plane along x and y (a ragged last tile covers the rest)
    int chunk;             // planes per block; blockIdx.y selects the chunk
    const int* entry_off;  // tiles_x tiles_y nz + 1 offsets into entries, by (tile, plane)
    const int2* entries;   // (special-cell index m, extended-tile position) of every source cell of the
                           // tile's extended cells, by tile then plane
};

// Where this thread's extended cell lies. Positions wrap periodically; a ragged last tile's core
// positions past the lattice's edge are not its own (the first tile steps those cells).
struct TileCell {
    int tile, bx, by;
    int cxy;   // x + nx y of the thread's extended cell
    bool core;
    int z0, z1;  // the block's planes
};

__host__ __device__ __forceinline__ bool tile_core(int local, int bx, int by, int nx, int ny) {
    const int ex = local % kTileEX, ey = local / kTileEX;
    return ex >= 1 && ex <= kTileTX && ey >= 1 && ey <= kTileTY && bx * kTileTX + ex - 1 < nx &&
           by * kTileTY + ey - 1 < ny;
}

__host__ __device__ __forceinline__ int tile_wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Lattice x (or y) of extended position e of tile b.
__host__ __device__ __forceinline__ int tile_coord(int b, int e, int t, int n) { return tile_wrap(b * t - 1 + e, n); }

__device__ __forceinline__ TileCell tile_cell(const Geometry& g, const TileArgs& T) {
    TileCell c;
    c.tile = blockIdx.x;
    c.by = blockIdx.x / T.tiles_x;
    c.bx = blockIdx.x - c.by * T.tiles_x;
    const int ex = threadIdx.x % kTileEX, ey = threadIdx.x / kTileEX;
    c.cxy = tile_coord(c.bx, ex, kTileTX, g.nx) + g.nx * tile_coord(c.by, ey, kTileTY, g.ny);
    c.core = tile_core(threadIdx.x, c.bx, c.by, g.nx, g.ny);
    c.z0 = blockIdx.y * T.chunk;
    c.z1 = min(c.z0 + T.chunk, g.nz);
    return c;
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
// Deterministic sum of v[0..count) into result[0] (one block, fixed order; result[1], [2] are 0).
int launch_sum_doubles(const double* v, int count, double* result, cudaStream_t st);

// Up to 8 independent device-to-device copies in one launch (sizes and addresses multiples of 4 B).
struct HaloChunk {
    const char* src;
    char* dst;
    long long bytes;
    int width;  // set by launch_halo_copy
};
struct HaloCopy {
    HaloChunk c[8];
    int count;
};
int launch_halo_copy(HaloCopy h, cudaStream_t st);
// Directions whose velocity has z component vz_sign (+1 or -1); returns their number.
int mm_halo_dirs(int vz_sign, int* dirs);
int hv_halo_dirs(int vz_sign, int* dirs);

// Batched step j: main launch over the first n_tiles tiles, source-cell launch over the first
// n_stiles special tiles. Returns the number of kernels enqueued.
int mm_launch_batch_step(const BatchLaunch& b, int j, int n_tiles, int n_stiles, cudaStream_t st);
int hv_launch_batch_step(const BatchLaunch& b, int j, int n_tiles, int n_stiles, cudaStream_t st);
// Resident blocks per SM of the main batched kernel for this configuration.
int mm_batch_occupancy(int storage, int block, bool rho);
int hv_batch_occupancy(int storage, int block);

// Adjoint launches (FP32 storage). adjoint: main launch over every cell not in special_mask, then
// the source cells. terminal: nu^T over the loss plane (nu_out must be zeroed first), and the
// first term of loss_plane. record_step: a forward step that also writes the adjoint record of
// every cell into a.rec.
int mm_launch_record_step(const StepArgs& a, cudaStream_t st);
// Two steps in one pass: aA is step t (fin = the current buffer), aB step t + 1 (fout = the other
// buffer); F describes the ring and the counters (zeroed by the caller). Returns launches.
int mm_launch_fused2(const StepArgs& aA, const StepArgs& aB, const FusedArgs& F, cudaStream_t st);
int hv_launch_fused2(const StepArgs& aA, const StepArgs& aB, const FusedArgs& F, cudaStream_t st);
// Resident blocks per SM of the two-step kernel.
int mm_fused2_occupancy(int storage, int media_mode);
int hv_fused2_occupancy(int storage, int media_mode);
// Two steps in one pass over shared-memory tiles: aA is step t, aB step t + 1; T the tiling. Returns
// launches. _occupancy: resident blocks per SM.
int mm_launch_tile2(const StepArgs& aA, const StepArgs& aB, const TileArgs& T, cudaStream_t st);
int hv_launch_tile2(const StepArgs& aA, const StepArgs& aB, const TileArgs& T, cudaStream_t st);
int mm_tile2_occupancy(int storage, int media_mode);
int hv_tile2_occupancy(int storage, int media_mode);
// The MM tiled pass that also writes both steps' adjoint records (aA.rec, aB.rec; FP32 storage only,
// else 0 launches).
int mm_launch_record_tile2(const StepArgs& aA, const StepArgs& aB, const TileArgs& T, cudaStream_t st);
int hv_launch_record_step(const StepArgs& a, cudaStream_t st);
int mm_launch_adjoint(const AdjointArgs& A, cudaStream_t st);
// Two MM backward steps in one pass over shared-memory tiles: A1 the step of nu^{n+1} -> nu^n (its
// nu_in is read), A2 the step nu^n -> nu^{n-1} (its nu_out is written); T the tiled pass's tiling.
int mm_launch_adjoint2(const AdjointArgs& A1, const AdjointArgs& A2, const TileArgs& T, cudaStream_t st);
int mm_launch_adjoint_terminal(const AdjointArgs& A, int n_plane, cudaStream_t st);
int hv_launch_adjoint(const AdjointArgs& A, cudaStream_t st);
int hv_launch_adjoint_terminal(const AdjointArgs& A, int n_plane, cudaStream_t st);

}  // namespace lbm
