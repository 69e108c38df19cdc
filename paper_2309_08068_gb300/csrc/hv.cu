// Modified Hauser-Verhey (HV) model kernels, arXiv 2309.08068 Section III.
//
// One thread updates one cell: 6 directions, each an electric vector e_i and a magnetic vector h_i
// (36 scalars), pulled as a 4-vector (e_x, e_y, e_z, h_x) and a 2-vector (h_y, h_z) from cell
// x - v_i (float4 + float2, or 8 + 4 bytes with 16-bit storage); arithmetic is FP32.
// Velocities in the Section III order: v1 = +x, v2 = +y, v3 = -x, v4 = -y, v5 = -z, v6 = +z.
//
// With tau = 1/2 the collision (eqs. equilibriumHV, CollisionHV, CollisionmodifiedHV) is
//   e_i' = 2 e_i^eq - e_i + T_i = D/3 - v_i x H - e_i - (J . v_i) v_i / 2
//   h_i' = 2 h_i^eq - h_i       = B/3 + v_i x E - h_i
// with D = sum e_i, B = sum h_i (eq. MacroscopicFieldsHV), E = D / eps, H = B / mu, eps = eps0 eps_r,
// mu = mu0 mu_r, and J = sigma E + J_ext. For v_i = s a (a a unit axis, s = +-1) the source term is
// -(J_a / 2) a whatever the sign s.
#include "lbm_internal.cuh"

namespace lbm {
namespace {

// Axis (0, 1, 2) and sign of v_i, i = 1..6.
constexpr int kHVAxis[6] = {0, 1, 0, 1, 2, 2};
constexpr int kHVSign[6] = {1, 1, -1, -1, -1, 1};

// s * (a x X) for the unit axis a.
template <int A, int S>
__device__ __forceinline__ float3 axis_cross(float3 X) {
    float3 r;
    if constexpr (A == 0) r = make_float3(0.f, -X.z, X.y);
    else if constexpr (A == 1) r = make_float3(X.z, 0.f, -X.x);
    else r = make_float3(-X.y, X.x, 0.f);
    if constexpr (S < 0) r = make_float3(-r.x, -r.y, -r.z);
    return r;
}

// Offset of the cell x - v_i.
template <int I>
__device__ __forceinline__ int pull_index(const Neighbourhood& h) {
    constexpr int a = kHVAxis[I], s = kHVSign[I];
    return shifted<a == 0 ? -s : 0, a == 1 ? -s : 0, a == 2 ? -s : 0>(h);
}

// Offset of the cell x + v_i.
template <int I>
__device__ __forceinline__ int push_index(const Neighbourhood& h) {
    constexpr int a = kHVAxis[I], s = kHVSign[I];
    return shifted<a == 0 ? s : 0, a == 1 ? s : 0, a == 2 ? s : 0>(h);
}

// 24-bit storage: in each of the two arrays the 6 planes of halves, then the 6 planes of correction
// bytes.
template <int S>
__device__ __forceinline__ void hv_pull(const StepArgs& a, const Neighbourhood& h, float4 (&e)[6], float2 (&hy)[6]) {
    if constexpr (S == kF24) {
        const size_t n6 = 6 * (size_t)a.g.n;
        const uint2* __restrict__ ehi = static_cast<const uint2*>(a.fin);
        const unsigned* __restrict__ elo = reinterpret_cast<const unsigned*>(ehi + n6);
        const unsigned* __restrict__ hhi = static_cast<const unsigned*>(a.fin2);
        const unsigned short* __restrict__ hlo = reinterpret_cast<const unsigned short*>(hhi + n6);
        static_for<0, 6>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            const size_t idx = (size_t)i * a.g.n + pull_index<i>(h);
            e[i] = F24::load4(ehi, elo, idx, a.inv_scale);
            hy[i] = F24::load2(hhi, hlo, idx, a.inv_scale);
        });
    } else {
        const auto* __restrict__ ein = static_cast<const typename Pack4<S>::T*>(a.fin);
        const auto* __restrict__ hin = static_cast<const typename Pack2<S>::T*>(a.fin2);
        static_for<0, 6>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            const int src = pull_index<i>(h);
            e[i] = Pack4<S>::load(ein + (size_t)i * a.g.n + src, a.inv_scale);
            hy[i] = Pack2<S>::load(hin + (size_t)i * a.g.n + src, a.inv_scale);
        });
    }
}

// Prefetch into L2 what the update of cell i will load: the populations hv_pull reads and the medium.
template <int S, int M>
__device__ __forceinline__ void hv_prefetch(const StepArgs& a, int i) {
    prefetch_media<M>(a.media, i);
    const auto* __restrict__ ein = static_cast<const typename Pack4<S>::T*>(a.fin);
    const auto* __restrict__ hin = static_cast<const typename Pack2<S>::T*>(a.fin2);
    const Neighbourhood h = neighbourhood(a.g, i);
    static_for<0, 6>([&](auto ic) {
        constexpr int k = decltype(ic)::value;
        const int src = pull_index<k>(h);
        prefetch_l2(ein + (size_t)k * a.g.n + src);
        prefetch_l2(hin + (size_t)k * a.g.n + src);
    });
}

template <int S>
__device__ __forceinline__ void hv_put(const StepArgs& a, int k, int i, float4 e, float2 hy) {
    if constexpr (S == kF24) {
        const size_t n6 = 6 * (size_t)a.g.n, idx = (size_t)k * a.g.n + i;
        uint2* __restrict__ ehi = static_cast<uint2*>(a.fout);
        unsigned* __restrict__ hhi = static_cast<unsigned*>(a.fout2);
        F24::store4(ehi, reinterpret_cast<unsigned*>(ehi + n6), idx, e, a.scale);
        F24::store2(hhi, reinterpret_cast<unsigned short*>(hhi + n6), idx, hy, a.scale);
    } else {
        auto* __restrict__ eout = static_cast<typename Pack4<S>::T*>(a.fout);
        auto* __restrict__ hout = static_cast<typename Pack2<S>::T*>(a.fout2);
        eout[(size_t)k * a.g.n + i] = Pack4<S>::pack(e, a.scale);
        hout[(size_t)k * a.g.n + i] = Pack2<S>::pack(hy, a.scale);
    }
}

struct HVFields {
    float3 D, B, E, H, J;
};

__device__ __forceinline__ HVFields hv_fields(const float4 (&e)[6], const float2 (&hy)[6], const MatCoef& mat,
                                              float3 jext) {
    HVFields F;
    // Pairwise sums ((1 + 2) + (3 + 4)) + (5 + 6) over the directions.
    float tx[6], ty[6], tz[6], ux[6], uy[6], uz[6];
    static_for<0, 6>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        tx[i] = e[i].x;
        ty[i] = e[i].y;
        tz[i] = e[i].z;
        ux[i] = e[i].w;
        uy[i] = hy[i].x;
        uz[i] = hy[i].y;
    });
    const float dx = pairwise_sum<0, 4>(tx) + pairwise_sum<4, 6>(tx);
    const float dy = pairwise_sum<0, 4>(ty) + pairwise_sum<4, 6>(ty);
    const float dz = pairwise_sum<0, 4>(tz) + pairwise_sum<4, 6>(tz);
    const float bx = pairwise_sum<0, 4>(ux) + pairwise_sum<4, 6>(ux);
    const float by = pairwise_sum<0, 4>(uy) + pairwise_sum<4, 6>(uy);
    const float bz = pairwise_sum<0, 4>(uz) + pairwise_sum<4, 6>(uz);
    const float eps = mat.c0.x, inv_eps = mat.c0.y, mu = mat.c0.z, inv_mu = mat.c0.w, sigma = mat.c1.x;
    F.D = make_float3(dx, dy, dz);
    F.B = make_float3(bx, by, bz);
    F.E = make_float3(div_rn(dx, eps, inv_eps), div_rn(dy, eps, inv_eps), div_rn(dz, eps, inv_eps));
    F.H = make_float3(div_rn(bx, mu, inv_mu), div_rn(by, mu, inv_mu), div_rn(bz, mu, inv_mu));
    F.J = make_float3(__fmaf_rn(sigma, F.E.x, jext.x), __fmaf_rn(sigma, F.E.y, jext.y),
                      __fmaf_rn(sigma, F.E.z, jext.z));
    return F;
}

constexpr float kInv3 = 1.0f / 3.0f;  // RN(1/3)
constexpr float kInv6 = 1.0f / 6.0f;  // RN(1/6)

__device__ __forceinline__ float3 sixth(float3 v) {
    return make_float3(div_rn(v.x, 6.f, kInv6), div_rn(v.y, 6.f, kInv6), div_rn(v.z, 6.f, kInv6));
}
// D / 6 with D = eps E.
__device__ __forceinline__ float3 hv_sixth_of_d(float3 E, const MatCoef& mat) {
    const float eps = mat.c0.x;
    return sixth(make_float3(eps * E.x, eps * E.y, eps * E.z));
}
// H = B / mu.
__device__ __forceinline__ float3 hv_h(float3 B, const MatCoef& mat) {
    const float mu = mat.c0.z, inv_mu = mat.c0.w;
    return make_float3(div_rn(B.x, mu, inv_mu), div_rn(B.y, mu, inv_mu), div_rn(B.z, mu, inv_mu));
}

// Where a step reads its populations and writes its results: the context's A/B buffers.
struct HVBuffers : NoStash {
    template <int S>
    __device__ void pull(const StepArgs& a, const Neighbourhood& h, float4 (&e)[6], float2 (&hy)[6]) const {
        hv_pull<S>(a, h, e, hy);
    }
    template <int S>
    __device__ void put(const StepArgs& a, int k, int i, float4 e, float2 hy) const {
        hv_put<S>(a, k, i, e, hy);
    }
};

// Update of cell i; m is its index in the special-cell list when kSpecial.
template <int S, int M, bool kSpecial, bool kRecord = false, class IO = HVBuffers>
__device__ __forceinline__ void hv_update(const StepArgs& a, int i, int m, const IO& io = IO{}) {
    const Neighbourhood h = neighbourhood(a.g, i);
    float4 e[6];
    float2 hy[6];
    io.template pull<S>(a, h, e, hy);
    if constexpr (IO::kStash)  // the h components wait in shared memory until the collision
        static_for<0, 6>([&](auto ic) {
            constexpr int k = decltype(ic)::value;
            io.stash_put(k, hy[k].x, hy[k].y);
            io.stash_put(6 + k, e[k].w, 0.f);  // h_x, which shares the float4 with e
        });
    const MatCoef mat = load_coef<kModelHV, M>(a.media, i, a.eps0, a.mu0);
    CellSource cs;
    float3 jext = make_float3(0.f, 0.f, 0.f);
    if constexpr (kSpecial) {
        cs = cell_source(a.sv, a.sc, m);
        jext = cs.J;
    }
    const HVFields F = hv_fields(e, hy, mat, jext);
    // Isotropic share of 2 e^eq and 2 h^eq: D / 3 and B / 3, correctly rounded (a multiplication by
    // RN(1/3) would bias every step by the same relative 3e-8 and drift D and B on long runs).
    const float3 q = make_float3(div_rn(F.D.x, 3.f, kInv3), div_rn(F.D.y, 3.f, kInv3), div_rn(F.D.z, 3.f, kInv3));
    const float3 p = make_float3(div_rn(F.B.x, 3.f, kInv3), div_rn(F.B.y, 3.f, kInv3), div_rn(F.B.z, 3.f, kInv3));
    static_for<0, 6>([&](auto ic) {
        constexpr int k = decltype(ic)::value;
        constexpr int A = kHVAxis[k], G = kHVSign[k];
        const float3 vH = axis_cross<A, G>(F.H);
        const float3 vE = axis_cross<A, G>(F.E);
        float3 eo = make_float3(q.x - vH.x - e[k].x, q.y - vH.y - e[k].y, q.z - vH.z - e[k].z);
        // eq. SourceTermHV: T_i = -(J . v_i) v_i / 2 = -(J_A / 2) along axis A.
        if constexpr (A == 0) eo.x -= 0.5f * F.J.x;
        else if constexpr (A == 1) eo.y -= 0.5f * F.J.y;
        else eo.z -= 0.5f * F.J.z;
        float hx = e[k].w, hyx = hy[k].x, hyy = hy[k].y;
        if constexpr (IO::kStash) {
            float unused;
            io.stash_get(k, hyx, hyy);
            io.stash_get(6 + k, hx, unused);
        }
        float3 ho = make_float3(p.x + vE.x - hx, p.y + vE.y - hyx, p.z + vE.z - hyy);
        if constexpr (kSpecial) {
            if (cs.imposed) {  // Appendix B "impose fields": f' = f_eq(E_imp, B_imp, J = 0)
                const float3 cH = axis_cross<A, G>(hv_h(cs.B, mat));
                const float3 cE = axis_cross<A, G>(cs.E);
                const float3 d6 = hv_sixth_of_d(cs.E, mat), b6 = sixth(cs.B);
                eo = make_float3(d6.x - 0.5f * cH.x, d6.y - 0.5f * cH.y, d6.z - 0.5f * cH.z);
                ho = make_float3(b6.x + 0.5f * cE.x, b6.y + 0.5f * cE.y, b6.z + 0.5f * cE.z);
            }
        }
        io.template put<S>(a, k, i, make_float4(eo.x, eo.y, eo.z, ho.x), make_float2(ho.y, ho.z));
    });
    if constexpr (kRecord) {  // what the adjoint of this step needs: E
        const int n = a.g.n;
        a.rec[i] = F.E.x;
        a.rec[n + i] = F.E.y;
        a.rec[2 * n + i] = F.E.z;
    }
}

// Two steps per pass (see FusedArgs): phase A streams the A/B buffers in once and writes the
// intermediate plane, phase B pulls from the intermediate planes (L2 loads) and streams the other
// A/B buffers out. The arithmetic is hv_update's, so the results equal two single steps bit for bit.
template <int S>
struct HVToRing : FusedStash {
    using T4 = typename Pack4<S>::T;
    using T2 = typename Pack2<S>::T;
    T4* plane;
    T2* plane2;
    int base, nxy;
    template <int S2>
    __device__ void pull(const StepArgs& a, const Neighbourhood& h, float4 (&e)[6], float2 (&hy)[6]) const {
        const T4* __restrict__ ein = static_cast<const T4*>(a.fin);
        const T2* __restrict__ hin = static_cast<const T2*>(a.fin2);
        static_for<0, 6>([&](auto ic) {
            constexpr int k = decltype(ic)::value;
            const int src = pull_index<k>(h);
            e[k] = Pack4<S>::unpack(__ldcs(ein + (size_t)k * a.g.n + src), a.inv_scale);
            hy[k] = Pack2<S>::unpack(__ldcs(hin + (size_t)k * a.g.n + src), a.inv_scale);
        });
    }
    template <int S2>
    __device__ void put(const StepArgs& a, int k, int i, float4 e, float2 hy) const {
        __stcg(plane + (size_t)k * nxy + (i - base), Pack4<S>::pack(e, a.scale));
        __stcg(plane2 + (size_t)k * nxy + (i - base), Pack2<S>::pack(hy, a.scale));
    }
};

template <int S>
struct HVFromRing : FusedStash {
    using T4 = typename Pack4<S>::T;
    using T2 = typename Pack2<S>::T;
    const T4* plane[3];  // slots of planes z - 1, z, z + 1
    const T2* plane2[3];
    int nxy;
    template <int S2>
    __device__ void pull(const StepArgs& a, const Neighbourhood& h, float4 (&e)[6], float2 (&hy)[6]) const {
        static_for<0, 6>([&](auto ic) {
            constexpr int k = decltype(ic)::value;
            constexpr int ax = kHVAxis[k], sg = kHVSign[k];
            constexpr int sx = ax == 0 ? -sg : 0, sy = ax == 1 ? -sg : 0, sz = ax == 2 ? -sg : 0;
            const int off = (int)((size_t)k * nxy) + h.xo[sx + 1] + h.yo[sy + 1];
            e[k] = Pack4<S>::unpack(__ldcg(plane[sz + 1] + off), a.inv_scale);
            hy[k] = Pack2<S>::unpack(__ldcg(plane2[sz + 1] + off), a.inv_scale);
        });
    }
    template <int S2>
    __device__ void put(const StepArgs& a, int k, int i, float4 e, float2 hy) const {
        T4* __restrict__ eout = static_cast<T4*>(a.fout);
        T2* __restrict__ hout = static_cast<T2*>(a.fout2);
        __stcs(eout + (size_t)k * a.g.n + i, Pack4<S>::pack(e, a.scale));
        __stcs(hout + (size_t)k * a.g.n + i, Pack2<S>::pack(hy, a.scale));
    }
};

template <int S, int M>
__global__ void __launch_bounds__(kFusedThreads, 3) hv_fused2_kernel(StepArgs aA, StepArgs aB, FusedArgs F) {
    using T4 = typename Pack4<S>::T;
    using T2 = typename Pack2<S>::T;
    __shared__ float2 s_stash[12 * kBlock];  // the h components, [slot][compute thread]
    const unsigned stash = fused_stash_slot(s_stash);
    const int nz = aA.g.nz, nxy = aA.g.nx * aA.g.ny;
    auto slot = [&](int p) -> T4* {
        if (p == 0) return static_cast<T4*>(F.lo);
        if (p == nz - 1) return static_cast<T4*>(F.hi);
        return static_cast<T4*>(F.ring) + (size_t)(p % F.R) * 6 * nxy;
    };
    auto slot2 = [&](int p) -> T2* {
        if (p == 0) return static_cast<T2*>(F.lo2);
        if (p == nz - 1) return static_cast<T2*>(F.hi2);
        return static_cast<T2*>(F.ring2) + (size_t)(p % F.R) * 6 * nxy;
    };
    auto describe = [&](const FusedItem& it, FusedDesc& d) {
        if (it.type == kPhaseA) {
            d.ptr[0] = slot(it.plane);
            d.ptr[1] = slot2(it.plane);
        } else {
            const int pm = (it.plane + nz - 1) % nz, pp = (it.plane + 1) % nz;
            d.ptr[0] = slot(pm);
            d.ptr[1] = slot(it.plane);
            d.ptr[2] = slot(pp);
            d.ptr[3] = slot2(pm);
            d.ptr[4] = slot2(it.plane);
            d.ptr[5] = slot2(pp);
        }
    };
    fused_loop(F, aA.g.nx, nxy, nz, describe, [&](const FusedDesc& d) {
        const int j = d.j, base = d.plane * nxy;
        if (d.type == kPhaseA) {
            const HVToRing<S> io{{stash}, static_cast<T4*>(d.ptr[0]), static_cast<T2*>(d.ptr[1]), base, nxy};
            const int end = min(base + (j + 1) * F.tile_cells, base + nxy);
            for (int i = base + j * F.tile_cells + threadIdx.x; i < end; i += kBlock)
                hv_update<S, M, false, false>(aA, i, 0, io);
            if (d.s_hi > d.s_lo) {  // the tile's source cells replace their ordinary update
                named_sync(kComputeBarrier, kBlock);
                for (int m = d.s_lo + threadIdx.x; m < d.s_hi; m += kBlock)
                    hv_update<S, M, true, false>(aA, aA.sv.cell[m], m, io);
            }
        } else {
            const HVFromRing<S> io{{stash},
                                   {static_cast<const T4*>(d.ptr[0]), static_cast<const T4*>(d.ptr[1]),
                                    static_cast<const T4*>(d.ptr[2])},
                                   {static_cast<const T2*>(d.ptr[3]), static_cast<const T2*>(d.ptr[4]),
                                    static_cast<const T2*>(d.ptr[5])},
                                   nxy};
            const int end = min(base + (j + 1) * F.tile_cells, base + nxy);
            for (int i = base + j * F.tile_cells + threadIdx.x; i < end; i += kBlock)
                hv_update<S, M, false, false>(aB, i, 0, io);
            if (d.s_hi > d.s_lo) {  // the tile's source cells replace their ordinary update
                named_sync(kComputeBarrier, kBlock);
                for (int m = d.s_lo + threadIdx.x; m < d.s_hi; m += kBlock)
                    hv_update<S, M, true, false>(aB, aB.sv.cell[m], m, io);
            }
        }
    });
}

// Two steps per pass over shared-memory tiles (see TileArgs). Directions by v_z: class 0 (v1 .. v4,
// in-plane), class 1 (v6 = +z), class 2 (v5 = -z).
__host__ __device__ constexpr int hv_zclass(int k) { return k < 4 ? 0 : (k == 5 ? 1 : 2); }
__host__ __device__ constexpr int hv_zrank(int k) { return k < 4 ? k : 0; }

// Direction planes of kTileThreads cells, for the 4-vectors and again for the 2-vectors: plane 0
// holds class 2 of the newest plane, 1-4 and 5-8 class 0 of the last two planes, 9-11 class 1 of
// the last three.
template <int S>
struct HVTile {
    using T4 = typename Pack4<S>::T;
    using T2 = typename Pack2<S>::T;
    static constexpr size_t kBytes = 12 * kTileThreads * (sizeof(T4) + sizeof(T2));
    T4* base4;
    T2* base2;
    __device__ int slot(int cls, int p) const {  // first direction plane of the class's slot, plane p >= -1
        return cls == 2 ? 0 : (cls == 0 ? 1 + 4 * ((p + 3) % 2) : 9 + (p + 3) % 3);
    }
};

template <int S>
struct HVToTile : NoStash {
    using T4 = typename Pack4<S>::T;
    using T2 = typename Pack2<S>::T;
    T4* base4;
    T2* base2;
    int slot[3];  // by class, for plane p
    int local;
    template <int S2>
    __device__ void pull(const StepArgs& a, const Neighbourhood& h, float4 (&e)[6], float2 (&hy)[6]) const {
        hv_pull<S>(a, h, e, hy);
    }
    template <int S2>
    __device__ void put(const StepArgs& a, int k, int, float4 ev, float2 hv) const {
        const int at = (slot[hv_zclass(k)] + hv_zrank(k)) * kTileThreads + local;
        base4[at] = Pack4<S>::pack(ev, a.scale);
        base2[at] = Pack2<S>::pack(hv, a.scale);
    }
};

template <int S>
struct HVFromTile : NoStash {
    using T4 = typename Pack4<S>::T;
    using T2 = typename Pack2<S>::T;
    const T4* base4;
    const T2* base2;
    int slot[3];  // class 0 of plane q, class 1 of q - 1, class 2 of q + 1
    int local;
    template <int S2>
    __device__ void pull(const StepArgs& a, const Neighbourhood&, float4 (&e)[6], float2 (&hy)[6]) const {
        static_for<0, 6>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            constexpr int ax = kHVAxis[k], sg = kHVSign[k];
            constexpr int vx = ax == 0 ? sg : 0, vy = ax == 1 ? sg : 0;
            const int at = (slot[hv_zclass(k)] + hv_zrank(k)) * kTileThreads + local - (vx + vy * kTileEX);
            e[k] = Pack4<S>::unpack(base4[at], a.inv_scale);
            hy[k] = Pack2<S>::unpack(base2[at], a.inv_scale);
        });
    }
    template <int S2>
    __device__ void put(const StepArgs& a, int k, int i, float4 ev, float2 hv) const {
        T4* __restrict__ eout = static_cast<T4*>(a.fout);
        T2* __restrict__ hout = static_cast<T2*>(a.fout2);
        __stcs(eout + (size_t)k * a.g.n + i, Pack4<S>::pack(ev, a.scale));
        __stcs(hout + (size_t)k * a.g.n + i, Pack2<S>::pack(hv, a.scale));
    }
};

template <int S, int M>
__global__ void __launch_bounds__(kTileThreads, S == kF32 ? 3 : 4) hv_tile2_kernel(StepArgs aA, StepArgs aB,
                                                                                    TileArgs T) {
    using T4 = typename Pack4<S>::T;
    using T2 = typename Pack2<S>::T;
    extern __shared__ __align__(16) unsigned char hv_tile_smem[];
    const HVTile<S> tile{reinterpret_cast<T4*>(hv_tile_smem),
                         reinterpret_cast<T2*>(hv_tile_smem + 12 * kTileThreads * sizeof(T4))};
    const int nz = aA.g.nz, nxy = aA.g.nx * aA.g.ny;
    const TileCell c = tile_cell(aA.g, T);
    const int* off = T.entry_off + (size_t)c.tile * nz;
    for (int p = c.z0 - 1; p <= c.z1; ++p) {
        const int pz = tile_wrap(p, nz);
        if (p < c.z1) hv_prefetch<S, M>(aA, tile_wrap(p + 1, nz) * nxy + c.cxy);  // as in mm_tile2_kernel
        {  // phase A: step t of the extended tile's cells of plane pz
            const HVToTile<S> io{{}, tile.base4, tile.base2, {tile.slot(0, p), tile.slot(1, p), tile.slot(2, p)},
                                 (int)threadIdx.x};
            hv_update<S, M, false, false>(aA, pz * nxy + c.cxy, 0, io);
            const int lo = off[pz], hi = off[pz + 1];
            if (hi > lo) {  // the source cells among them replace their ordinary update
                __syncthreads();
                for (int k = lo + threadIdx.x; k < hi; k += kTileThreads) {
                    const int2 e = T.entries[k];
                    const HVToTile<S> sio{{}, io.base4, io.base2, {io.slot[0], io.slot[1], io.slot[2]}, e.y};
                    hv_update<S, M, true, false>(aA, aA.sv.cell[e.x], e.x, sio);
                }
            }
        }
        __syncthreads();
        if (p > c.z0) {  // phase B: step t + 1 of the tile's own cells of plane q = p - 1
            const int q = p - 1;
            const HVFromTile<S> io{{}, tile.base4, tile.base2, {tile.slot(0, q), tile.slot(1, q - 1), tile.slot(2, q + 1)},
                                   (int)threadIdx.x};
            if (c.core) hv_update<S, M, false, false>(aB, q * nxy + c.cxy, 0, io);
            const int lo = off[q], hi = off[q + 1];
            if (hi > lo) {
                __syncthreads();
                for (int k = lo + threadIdx.x; k < hi; k += kTileThreads) {
                    const int2 e = T.entries[k];
                    if (!tile_core(e.y, c.bx, c.by, aA.g.nx, aA.g.ny)) continue;
                    const HVFromTile<S> sio{{}, io.base4, io.base2, {io.slot[0], io.slot[1], io.slot[2]}, e.y};
                    hv_update<S, M, true, false>(aB, aB.sv.cell[e.x], e.x, sio);
                }
            }
        }
        __syncthreads();
    }
}

// The block's source cells are recomputed at the end (block_source_cells). 4 resident blocks (64
// registers); 3 for 24-bit storage, whose decoding would spill at 64.
template <int S, int M>
__global__ void __launch_bounds__(kBlock, S == kF24 ? 3 : 4) hv_step_kernel(StepArgs a) {
    const int i = a.cell_begin + blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.cell_end) hv_update<S, M, false>(a, i, 0);
    block_source_cells(a.sv, blockIdx.x, [&](int c, int m) { hv_update<S, M, true>(a, c, m); });
}

// Equilibria for fields E, B and J = 0 (Appendix B initialisation), stored so that cell x pulls
// them at the next step: direction i at y holds the equilibrium of cell y + v_i.
template <int S, int M>
__global__ void __launch_bounds__(kBlock) hv_init_kernel(StepArgs a, const float* __restrict__ E,
                                                         const float* __restrict__ B) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= a.g.n) return;
    const int n = a.g.n;
    const Neighbourhood h = neighbourhood(a.g, y);
    static_for<0, 6>([&](auto ic) {
        constexpr int k = decltype(ic)::value;
        constexpr int A = kHVAxis[k], G = kHVSign[k];
        const int x = push_index<k>(h);
        const MatCoef mat = load_coef<kModelHV, M>(a.media, x, a.eps0, a.mu0);
        const float3 Ex = make_float3(__ldg(&E[x]), __ldg(&E[n + x]), __ldg(&E[2 * n + x]));
        const float3 Bx = make_float3(__ldg(&B[x]), __ldg(&B[n + x]), __ldg(&B[2 * n + x]));
        const float3 cH = axis_cross<A, G>(hv_h(Bx, mat));
        const float3 cE = axis_cross<A, G>(Ex);
        const float3 d6 = hv_sixth_of_d(Ex, mat), b6 = sixth(Bx);
        // e^eq = (D - 3 v x B / mu) / 6 = D/6 - (v x H)/2;  h^eq = (B + 3 v x D / eps) / 6 = B/6 + (v x E)/2
        hv_put<S>(a, k, y,
                  make_float4(d6.x - 0.5f * cH.x, d6.y - 0.5f * cH.y, d6.z - 0.5f * cH.z, b6.x + 0.5f * cE.x),
                  make_float2(b6.y + 0.5f * cE.y, b6.z + 0.5f * cE.z));
    });
}

template <int S, int M, bool kSpecial>
__global__ void __launch_bounds__(kBlock) hv_fields_kernel(StepArgs a, FieldsOut out) {
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
    float4 e[6];
    float2 hy[6];
    hv_pull<S>(a, h, e, hy);
    const MatCoef mat = load_coef<kModelHV, M>(a.media, i, a.eps0, a.mu0);
    float3 jext = make_float3(0.f, 0.f, 0.f);
    if constexpr (kSpecial) jext = cell_source(a.sv, a.sc, m).J;
    const HVFields F = hv_fields(e, hy, mat, jext);
    auto put = [&](float* p, float3 v) {
        if (p) {
            p[i] = v.x;
            p[n + i] = v.y;
            p[2 * n + i] = v.z;
        }
    };
    put(out.E, F.E);
    put(out.B, F.B);
    put(out.D, F.D);
    put(out.H, F.H);
    put(out.J, F.J);
}

// Canonical layout out[k * n + x], k = r*18 + (i-1)*3 + c.
template <int S>
__global__ void __launch_bounds__(kBlock) hv_get_kernel(StepArgs a, float* __restrict__ out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.g.n) return;
    const int n = a.g.n;
    const Neighbourhood h = neighbourhood(a.g, x);
    float4 e[6];
    float2 hy[6];
    hv_pull<S>(a, h, e, hy);
    static_for<0, 6>([&](auto ic) {
        constexpr int k = decltype(ic)::value;
        out[(size_t)(3 * k + 0) * n + x] = e[k].x;
        out[(size_t)(3 * k + 1) * n + x] = e[k].y;
        out[(size_t)(3 * k + 2) * n + x] = e[k].z;
        out[(size_t)(18 + 3 * k + 0) * n + x] = e[k].w;
        out[(size_t)(18 + 3 * k + 1) * n + x] = hy[k].x;
        out[(size_t)(18 + 3 * k + 2) * n + x] = hy[k].y;
    });
}

template <int S>
__global__ void __launch_bounds__(kBlock) hv_set_kernel(StepArgs a, const float* __restrict__ in) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= a.g.n) return;
    const int n = a.g.n;
    const Neighbourhood h = neighbourhood(a.g, y);
    static_for<0, 6>([&](auto ic) {
        constexpr int k = decltype(ic)::value;
        const int x = push_index<k>(h);
        hv_put<S>(a, k, y,
                  make_float4(in[(size_t)(3 * k) * n + x], in[(size_t)(3 * k + 1) * n + x],
                              in[(size_t)(3 * k + 2) * n + x], in[(size_t)(18 + 3 * k) * n + x]),
                  make_float2(in[(size_t)(19 + 3 * k) * n + x], in[(size_t)(20 + 3 * k) * n + x]));
    });
}

// Per-block partial sums of (1/2)(E.D + B.H) and sum f^2 (E does not depend on J_ext in HV, so no
// source-cell correction is needed).
template <int S, int M>
__global__ void __launch_bounds__(kBlock) hv_reduce_kernel(StepArgs a, double* __restrict__ partials) {
    double w = 0.0, f2 = 0.0;
    for (int i = a.cell_begin + blockIdx.x * blockDim.x + threadIdx.x; i < a.cell_end; i += gridDim.x * blockDim.x) {
        const Neighbourhood h = neighbourhood(a.g, i);
        float4 e[6];
        float2 hy[6];
        hv_pull<S>(a, h, e, hy);
        const MatCoef mat = load_coef<kModelHV, M>(a.media, i, a.eps0, a.mu0);
        const HVFields F = hv_fields(e, hy, mat, make_float3(0.f, 0.f, 0.f));
        w += 0.5 * ((double)F.E.x * F.D.x + (double)F.E.y * F.D.y + (double)F.E.z * F.D.z +
                    (double)F.B.x * F.H.x + (double)F.B.y * F.H.y + (double)F.B.z * F.H.z);
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k)
            s += (double)e[k].x * e[k].x + (double)e[k].y * e[k].y + (double)e[k].z * e[k].z +
                 (double)e[k].w * e[k].w + (double)hy[k].x * hy[k].x + (double)hy[k].y * hy[k].y;
        f2 += s;
    }
    block_sum3_store(w, f2, 0.0, partials + 3 * blockIdx.x);
}

// Batched step j of several lattices (see mm_batch_kernel).
template <int S, int BLOCK>
__global__ void __launch_bounds__(BLOCK) hv_batch_kernel(const BatchLattice* __restrict__ lat,
                                                         const BatchTile* __restrict__ tiles, int n_tiles, int j) {
    for (int b = blockIdx.x; b < n_tiles; b += gridDim.x) {
        const BatchTile tile = tiles[b];
        const BatchLattice* L = &lat[tile.lattice];
        const int i = tile.begin + threadIdx.x;
        if (j >= L->steps || i >= L->base.g.n) continue;
        const StepArgs a = batch_args(L, j);
        switch (a.media_mode) {
            case kUniform: hv_update<S, kUniform, false>(a, i, 0); break;
            case kTable: hv_update<S, kTable, false>(a, i, 0); break;
            default: hv_update<S, kPerCell, false>(a, i, 0); break;
        }
    }
}

template <int S>
__global__ void __launch_bounds__(kBlock) hv_batch_special_kernel(const BatchLattice* __restrict__ lat,
                                                                  const BatchTile* __restrict__ tiles, int j) {
    const BatchTile tile = tiles[blockIdx.x];
    const BatchLattice* L = &lat[tile.lattice];
    const int m = tile.begin + threadIdx.x;
    if (j >= L->steps || m >= L->base.sv.n_special) return;
    StepArgs a = batch_args(L, j);
    batch_sources(L, j, a);
    const int i = a.sv.cell[m];
    switch (a.media_mode) {
        case kUniform: hv_update<S, kUniform, true>(a, i, m); break;
        case kTable: hv_update<S, kTable, true>(a, i, m); break;
        default: hv_update<S, kPerCell, true>(a, i, m); break;
    }
}

template <int M>
__global__ void __launch_bounds__(kBlock) hv_record_kernel(StepArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.g.n) hv_update<kF32, M, false, true>(a, i, 0);
    block_source_cells(a.sv, blockIdx.x, [&](int c, int m) { hv_update<kF32, M, true, true>(a, c, m); });
}

// ---------------------------------------------------------------------------------------------
// Adjoint of one HV step. With adjoints e_i^, h_i^ of the post-collision vectors, the transpose of
// e_i' = D/3 - v_i x H - e_i - (J . v_i) v_i / 2 and h_i' = B/3 + v_i x E - h_i is
//   gH = sum_i v_i x e_i^,   gE = sum_i h_i^ x v_i + sigma gJ,   gJ_a = -(1/2) sum_{i on axis a} e_i^_a,
//   gD = sum_i e_i^ / 3 + gE / eps,   gB = sum_i h_i^ / 3 + gH / mu,
//   nu(e_i) = gD - e_i^,   nu(h_i) = gB - h_i^,
//   dL/d eps_r += -gE . E / eps_r   (E = D / (eps0 eps_r)),   dL/d sigma += gJ . E.
// Imposed cells output f_eq(E_imp, B_imp, 0), where D_imp = eps0 eps_r E_imp: nothing flows back
// to f, and d e_i' / d eps_r = eps0 E_imp / 6. The plane loss |E|^2 adds 2E to gE.
template <int M, bool kSpecial, bool kTerminal>
__device__ __forceinline__ void hv_adjoint_cell(const AdjointArgs& A, int i, int m) {
    const StepArgs& a = A.a;
    const int n = a.g.n;
    const Neighbourhood h = neighbourhood(a.g, i);
    const MatCoef mat = load_coef<kModelHV, M>(a.media, i, a.eps0, a.mu0);
    CellSource cs;
    bool imposed = false;
    if constexpr (kSpecial) {
        cs = cell_source(a.sv, a.sc, m);
        imposed = cs.imposed;
    }
    // Every load is issued up front: the source-cell mask of the main launch only gates the stores,
    // so it adds no round trip before the others.
    const bool skip = !kSpecial && !kTerminal && A.special_mask[i] != 0;
    const float geps_old = __ldg(&A.grad_eps[i]), gsig_old = A.grad_sigma ? __ldg(&A.grad_sigma[i]) : 0.f;
    // E of f^n: from the forward step's record, or (terminal) from the final state
    float3 E;
    if constexpr (kTerminal) {
        float4 e[6];
        float2 hy[6];
        hv_pull<kF32>(a, h, e, hy);
        E = hv_fields(e, hy, mat, make_float3(0.f, 0.f, 0.f)).E;
    } else {
        E = make_float3(__ldg(&a.rec[i]), __ldg(&a.rec[n + i]), __ldg(&a.rec[2 * n + i]));
    }
    struct {
        float3 E;
    } F{E};
    const float inv_eps = mat.c0.y, inv_mu = mat.c0.w, sigma = mat.c1.x, er = mat.c1.y;
    float4 le[6];
    float2 lh[6];
    static_for<0, 6>([&](auto ic) {
        constexpr int k = decltype(ic)::value;
        if constexpr (kTerminal) {
            le[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            lh[k] = make_float2(0.f, 0.f);
        } else {
            const int dst = push_index<k>(h);
            le[k] = __ldg(static_cast<const float4*>(A.nu_in) + (size_t)k * n + dst);
            lh[k] = __ldg(static_cast<const float2*>(A.nu_in2) + (size_t)k * n + dst);
        }
    });
    float3 Se = make_float3(0.f, 0.f, 0.f), Sh = Se, gH = Se, gE = Se, gJ = Se;
    float geps_imposed = 0.f;
    if (!imposed) {
        static_for<0, 6>([&](auto ic) {
            constexpr int k = decltype(ic)::value;
            constexpr int AX = kHVAxis[k], G = kHVSign[k];
            const float3 ek = make_float3(le[k].x, le[k].y, le[k].z);
            const float3 hk = make_float3(le[k].w, lh[k].x, lh[k].y);
            Se = make_float3(Se.x + ek.x, Se.y + ek.y, Se.z + ek.z);
            Sh = make_float3(Sh.x + hk.x, Sh.y + hk.y, Sh.z + hk.z);
            const float3 ve = axis_cross<AX, G>(ek);  // v_k x e_k^
            const float3 vh = axis_cross<AX, G>(hk);  // v_k x h_k^ = -(h_k^ x v_k)
            gH = make_float3(gH.x + ve.x, gH.y + ve.y, gH.z + ve.z);
            gE = make_float3(gE.x - vh.x, gE.y - vh.y, gE.z - vh.z);
            if constexpr (AX == 0) gJ.x -= 0.5f * ek.x;
            else if constexpr (AX == 1) gJ.y -= 0.5f * ek.y;
            else gJ.z -= 0.5f * ek.z;
        });
        gE = make_float3(__fmaf_rn(sigma, gJ.x, gE.x), __fmaf_rn(sigma, gJ.y, gE.y), __fmaf_rn(sigma, gJ.z, gE.z));
    } else if constexpr (kSpecial) {
        const float3 dE = make_float3(div_rn(a.eps0 * cs.E.x, 6.f, kInv6), div_rn(a.eps0 * cs.E.y, 6.f, kInv6),
                                      div_rn(a.eps0 * cs.E.z, 6.f, kInv6));
        static_for<0, 6>([&](auto ic) {
            constexpr int k = decltype(ic)::value;
            geps_imposed += le[k].x * dE.x + le[k].y * dE.y + le[k].z * dE.z;
        });
    }
    if (A.loss_active && in_plane(h, a.g, A.plane_axis, A.plane_index)) {  // |E|^2 of time n
        gE = make_float3(__fmaf_rn(2.f, F.E.x, gE.x), __fmaf_rn(2.f, F.E.y, gE.y), __fmaf_rn(2.f, F.E.z, gE.z));
        add_plane_loss<kTerminal>(A, h, F.E);
    }
    const float3 gD = make_float3(__fmaf_rn(gE.x, inv_eps, div_rn(Se.x, 3.f, kInv3)),
                                  __fmaf_rn(gE.y, inv_eps, div_rn(Se.y, 3.f, kInv3)),
                                  __fmaf_rn(gE.z, inv_eps, div_rn(Se.z, 3.f, kInv3)));
    const float3 gB = make_float3(__fmaf_rn(gH.x, inv_mu, div_rn(Sh.x, 3.f, kInv3)),
                                  __fmaf_rn(gH.y, inv_mu, div_rn(Sh.y, 3.f, kInv3)),
                                  __fmaf_rn(gH.z, inv_mu, div_rn(Sh.z, 3.f, kInv3)));
    if (skip) return;  // a source cell: the second launch writes it
    float4* eout = static_cast<float4*>(A.nu_out);
    float2* hout = static_cast<float2*>(A.nu_out2);
    static_for<0, 6>([&](auto ic) {
        constexpr int k = decltype(ic)::value;
        float4 o;
        float2 p;
        if (imposed) {
            o = make_float4(gD.x, gD.y, gD.z, gB.x);
            p = make_float2(gB.y, gB.z);
        } else {
            o = make_float4(gD.x - le[k].x, gD.y - le[k].y, gD.z - le[k].z, gB.x - le[k].w);
            p = make_float2(gB.y - lh[k].x, gB.z - lh[k].y);
        }
        eout[(size_t)k * n + i] = o;
        hout[(size_t)k * n + i] = p;
    });
    // explicit fused multiply-adds wherever a product meets a sum (the same bits in every kernel)
    const float gEdotE = __fmaf_rn(gE.z, F.E.z, __fmaf_rn(gE.y, F.E.y, __fmul_rn(gE.x, F.E.x)));
    A.grad_eps[i] = geps_old + (geps_imposed - div_rn(gEdotE, er, 1.f / er));
    if (A.grad_sigma)
        A.grad_sigma[i] = gsig_old + __fmaf_rn(gJ.z, F.E.z, __fmaf_rn(gJ.y, F.E.y, __fmul_rn(gJ.x, F.E.x)));
}

// Source cells (skipped by the ordinary update through the mask) are stepped back at the end of
// their block (block_source_cells).
template <int M>
__global__ void __launch_bounds__(kBlock) hv_adjoint_kernel(AdjointArgs A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < A.a.g.n) hv_adjoint_cell<M, false, false>(A, i, 0);
    block_source_cells(A.a.sv, blockIdx.x, [&](int c, int m) { hv_adjoint_cell<M, true, false>(A, c, m); });
}

template <int M>
__global__ void __launch_bounds__(kBlock) hv_adjoint_terminal_kernel(AdjointArgs A, int n_plane) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_plane) return;
    hv_adjoint_cell<M, false, true>(A, plane_cell(A.a.g, A.plane_axis, A.plane_index, k), 0);
}

}  // namespace

int hv_launch_step(const StepArgs& a, cudaStream_t st) {
    int launched = 0;
    with_storage(a.storage, [&](auto sc) {
        with_media(a.media_mode, [&](auto mc) {
            constexpr int S = decltype(sc)::value, M = decltype(mc)::value;
            hv_step_kernel<S, M><<<blocks_for(a.cell_end - a.cell_begin), kBlock, 0, st>>>(a);
            launched = 1;
        });
    });
    return launched;
}

int hv_launch_init(const StepArgs& a, const float* E, const float* B, cudaStream_t st) {
    with_storage(a.storage, [&](auto sc) {
        with_media(a.media_mode, [&](auto mc) {
            constexpr int S = decltype(sc)::value, M = decltype(mc)::value;
            hv_init_kernel<S, M><<<blocks_for(a.g.n), kBlock, 0, st>>>(a, E, B);
        });
    });
    return 1;
}

int hv_launch_fields(const StepArgs& a, FieldsOut out, cudaStream_t st) {
    int launched = 0;
    with_storage(a.storage, [&](auto sc) {
        with_media(a.media_mode, [&](auto mc) {
            constexpr int S = decltype(sc)::value, M = decltype(mc)::value;
            hv_fields_kernel<S, M, false><<<blocks_for(a.g.n), kBlock, 0, st>>>(a, out);
            launched = 1;
            if (a.sv.n_special > 0) {
                hv_fields_kernel<S, M, true><<<blocks_for(a.sv.n_special), kBlock, 0, st>>>(a, out);
                launched = 2;
            }
        });
    });
    return launched;
}

int hv_launch_get(const StepArgs& a, float* out, cudaStream_t st) {
    with_storage(a.storage, [&](auto sc) {
        constexpr int S = decltype(sc)::value;
        hv_get_kernel<S><<<blocks_for(a.g.n), kBlock, 0, st>>>(a, out);
    });
    return 1;
}

int hv_launch_set(const StepArgs& a, const float* in, cudaStream_t st) {
    with_storage(a.storage, [&](auto sc) {
        constexpr int S = decltype(sc)::value;
        hv_set_kernel<S><<<blocks_for(a.g.n), kBlock, 0, st>>>(a, in);
    });
    return 1;
}

int hv_launch_reduce(const StepArgs& a, double* partials, int n_blocks, double* result, cudaStream_t st) {
    with_storage(a.storage, [&](auto sc) {
        with_media(a.media_mode, [&](auto mc) {
            constexpr int S = decltype(sc)::value, M = decltype(mc)::value;
            hv_reduce_kernel<S, M><<<n_blocks, kBlock, 0, st>>>(a, partials);
        });
    });
    return 1 + launch_reduce_partials(partials, n_blocks, result, st);
}

int hv_launch_batch_step(const BatchLaunch& b, int j, int n_tiles, int n_stiles, cudaStream_t st) {
    int launched = 0;
    with_storage(b.storage, [&](auto sc) {
        constexpr int S = decltype(sc)::value;
        if (n_tiles > 0) {
            const int grid = b.grid_cap > 0 ? (n_tiles < b.grid_cap ? n_tiles : b.grid_cap) : n_tiles;
            if (b.block == 128) hv_batch_kernel<S, 128><<<grid, 128, 0, st>>>(b.lat, b.tiles, n_tiles, j);
            else hv_batch_kernel<S, 256><<<grid, 256, 0, st>>>(b.lat, b.tiles, n_tiles, j);
            ++launched;
        }
        if (n_stiles > 0) {
            hv_batch_special_kernel<S><<<n_stiles, kBlock, 0, st>>>(b.lat, b.stiles, j);
            ++launched;
        }
    });
    return launched;
}

int hv_batch_occupancy(int storage, int block) {
    int blocks = 0;
    with_storage(storage, [&](auto sc) {
        constexpr int S = decltype(sc)::value;
        if (block == 128) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, hv_batch_kernel<S, 128>, 128, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, hv_batch_kernel<S, 256>, 256, 0);
    });
    return blocks;
}

int hv_launch_adjoint(const AdjointArgs& A, cudaStream_t st) {
    int launched = 0;
    with_media(A.a.media_mode, [&](auto mc) {
        constexpr int M = decltype(mc)::value;
        hv_adjoint_kernel<M><<<blocks_for(A.a.g.n), kBlock, 0, st>>>(A);
        launched = 1;
    });
    return launched;
}

int hv_launch_adjoint_terminal(const AdjointArgs& A, int n_plane, cudaStream_t st) {
    with_media(A.a.media_mode, [&](auto mc) {
        constexpr int M = decltype(mc)::value;
        hv_adjoint_terminal_kernel<M><<<blocks_for(n_plane), kBlock, 0, st>>>(A, n_plane);
    });
    return 1;
}

int hv_fused2_occupancy(int storage, int media_mode) {
    int blocks = 0;
    with_pass_storage(storage, [&](auto sc) {
        with_media(media_mode, [&](auto mc) {
            constexpr int S = decltype(sc)::value, M = decltype(mc)::value;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, hv_fused2_kernel<S, M>, kFusedThreads, 0);
        });
    });
    return blocks;
}

int hv_launch_fused2(const StepArgs& aA, const StepArgs& aB, const FusedArgs& F, cudaStream_t st) {
    if (aA.storage == kF24) return 0;  // no 24-bit form of the passes
    const int grid = fused_grid(hv_fused2_occupancy(aA.storage, aA.media_mode));
    with_pass_storage(aA.storage, [&](auto sc) {
        with_media(aA.media_mode, [&](auto mc) {
            constexpr int S = decltype(sc)::value, M = decltype(mc)::value;
            hv_fused2_kernel<S, M><<<grid, kFusedThreads, 0, st>>>(aA, aB, F);
        });
    });
    return 1;
}

template <int S, int M>
void hv_tile2_prepare() {
    static bool done = false;  // the attribute is a property of the kernel: set it once per process
    if (!done) {
        cudaFuncSetAttribute(hv_tile2_kernel<S, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HVTile<S>::kBytes);
        done = true;
    }
}

int hv_tile2_occupancy(int storage, int media_mode) {
    int blocks = 0;
    with_pass_storage(storage, [&](auto sc) {
        with_media(media_mode, [&](auto mc) {
            constexpr int S = decltype(sc)::value, M = decltype(mc)::value;
            hv_tile2_prepare<S, M>();
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, hv_tile2_kernel<S, M>, kTileThreads,
                                                          HVTile<S>::kBytes);
        });
    });
    return blocks;
}

int hv_launch_tile2(const StepArgs& aA, const StepArgs& aB, const TileArgs& T, cudaStream_t st) {
    if (aA.storage == kF24) return 0;  // no 24-bit form of the passes
    const dim3 grid(T.tiles_x * T.tiles_y, (aA.g.nz + T.chunk - 1) / T.chunk);
    with_pass_storage(aA.storage, [&](auto sc) {
        with_media(aA.media_mode, [&](auto mc) {
            constexpr int S = decltype(sc)::value, M = decltype(mc)::value;
            hv_tile2_prepare<S, M>();
            hv_tile2_kernel<S, M><<<grid, kTileThreads, HVTile<S>::kBytes, st>>>(aA, aB, T);
        });
    });
    return 1;
}

int hv_halo_dirs(int vz_sign, int* dirs) {
    int k = 0;
    for (int d = 0; d < 6; ++d)
        if (kHVAxis[d] == 2 && kHVSign[d] == vz_sign) dirs[k++] = d;
    return k;
}

int hv_launch_record_step(const StepArgs& a, cudaStream_t st) {
    int launched = 0;
    with_media(a.media_mode, [&](auto mc) {
        constexpr int M = decltype(mc)::value;
        hv_record_kernel<M><<<blocks_for(a.g.n), kBlock, 0, st>>>(a);
        launched = 1;
    });
    return launched;
}

}  // namespace lbm
