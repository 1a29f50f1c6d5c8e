// Packed FP32 pair arithmetic, the paired-cell face flux and the
// shared-memory copy helpers used by the paired-cell stage kernels (one
// stage per pass, and two stages per pass).
#pragma once

#include "rkl_device.cuh"

namespace rkl {
namespace x2 {

// --------------------------------------------------------------------------
// packed FP32 pair arithmetic

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    unsigned long long r, x = *reinterpret_cast<unsigned long long*>(&a),
                          y = *reinterpret_cast<unsigned long long*>(&b);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
    return *reinterpret_cast<float2*>(&r);
}
__device__ __forceinline__ float2 bc2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 sqrt2(float2 a) { return make_float2(dsqrt<float>(a.x), dsqrt<float>(a.y)); }

// Normal flux on a pair of faces (the packed form of face_flux).
template <bool SP, bool SAT>
__device__ __forceinline__ float2 face2(float2 TL, float2 TR, float2 gn, float2 g1, float2 g2, float2 bn, float2 b1,
                                        float2 b2, const KPhys<float>& p)
{
    const float2 Tf = mul2(bc2(0.5f), add2(TL, TR));
    float2 nk;                                    // -kappa_par at the face
    if (SP) nk = mul2(mul2(bc2(-p.kappa0), mul2(Tf, Tf)), sqrt2(Tf));
    else nk = bc2(-p.kappa0);
    const float2 nkp = mul2(bc2(p.kperp), nk);    // -kappa_perp
    const float2 bdg = fma2(bn, gn, fma2(b1, g1, mul2(b2, g2)));
    float2 Fn = fma2(mul2(nk, bn), bdg, mul2(nkp, gn));
    if (SAT) {
        const float2 F1 = fma2(mul2(nk, b1), bdg, mul2(nkp, g1));
        const float2 F2 = fma2(mul2(nk, b2), bdg, mul2(nkp, g2));
        const float2 F2s = fma2(Fn, Fn, fma2(F1, F1, mul2(F2, F2)));
        const float2 Fmag = sqrt2(F2s);
        float2 Tq = Tf;
        if (p.upwind) {
            Tq.x = Fn.x >= 0.f ? TL.x : TR.x;
            Tq.y = Fn.y >= 0.f ? TL.y : TR.y;
        }
        const float2 q = mul2(mul2(bc2(p.q0), Tq), sqrt2(Tq));
        const float2 den = add2(q, Fmag);
        Fn = make_float2(ddiv<float>(q.x, den.x) * Fn.x, ddiv<float>(q.y, den.y) * Fn.y);
    }
    return Fn;
}

// Constants of the folded face flux below.  With Bn = b_L,n + b_R,n (a sum,
// not the average) and Ts = T_L + T_R, the flux of Eq. qN is
//   F = -kappa_par(Ts / 2) / 4 * (Bn (B . g) + 4 (kappa_perp / kappa_par) gn),
// so the halves of the face averages and the whole prefactor become one
// constant per launch, and face2s returns F / fscale (the divergence absorbs
// fscale).
//
// Saturation (Eq. qsat) blends F with q = q0 (Ts / 2)^1.5 as F q / (q + |F|).
// Write F = nk Ts^2.5 V_n (Spitzer; nk Ts^0 for a constant kappa) with
// V = (X, Y1, Y2) the bracket above for the three flux components.  When q
// is taken at the face temperature, Ts^1.5 cancels between q and |F|:
//   F_sat / nk = Ts^2.5 X / (1 + s Ts |V|)              (Spitzer)
//   F_sat / nk = Ts^1.5 X / (Ts^1.5 + s |V|)            (constant kappa)
// with s = -nk / (q0 2^-1.5), so the blend costs |V| and one division and
// no separate q.  The upwind choice of q (the donor cell's temperature)
// does not cancel; that form returns F itself and fscale = 1.
struct FaceK {
    float nk;         // -kappa_par0 / 4 (x 2^-2.5 under Spitzer: (Ts / 2)^2.5)
    float kp4;        // 4 kappa_perp / kappa_par
    float fscale;     // true flux = fscale x returned value
    float sat;        // s above (saturation at the face temperature)
};

template <bool SP, bool SAT>
__device__ __forceinline__ FaceK face_consts(const KPhys<float>& p)
{
    FaceK k;
    k.nk = -0.25f * p.kappa0 * (SP ? 0.17677669529663688f : 1.f);    // 2^-2.5
    k.kp4 = 4.f * p.kperp;
    k.fscale = (SAT && p.upwind) ? 1.f : k.nk;
    k.sat = SAT ? -k.nk / (p.q0 * 0.35355339059327373f) : 0.f;       // 2^-1.5
    return k;
}

// KP0: kappa_perp = 0 known at compile time; the perpendicular terms
// (fma with a zero product) drop out, which for finite operands gives the
// same bits.
template <bool SP, bool SAT, bool KP0 = false>
__device__ __forceinline__ float2 face2s(float2 TL, float2 TR, float2 gn, float2 g1, float2 g2, float2 Bn, float2 B1,
                                         float2 B2, const FaceK& k, const KPhys<float>& p)
{
    const float2 Ts = add2(TL, TR);
    const float2 bdg = fma2(Bn, gn, fma2(B1, g1, mul2(B2, g2)));
    const float2 X = KP0 ? mul2(Bn, bdg) : fma2(Bn, bdg, mul2(bc2(k.kp4), gn));
    if (!SAT) {
        if (SP) return mul2(mul2(mul2(Ts, Ts), sqrt2(Ts)), X);
        return X;
    }
    const float2 sTs = sqrt2(Ts);
    // |V|^2, one transverse component at a time
    float2 V2 = mul2(X, X);
    const float2 Y1 = KP0 ? mul2(B1, bdg) : fma2(B1, bdg, mul2(bc2(k.kp4), g1));
    V2 = fma2(Y1, Y1, V2);
    const float2 Y2 = KP0 ? mul2(B2, bdg) : fma2(B2, bdg, mul2(bc2(k.kp4), g2));
    V2 = fma2(Y2, Y2, V2);
    if (!p.upwind) {
        const float2 Vm = sqrt2(V2);
        float2 num, den;
        if (SP) {
            num = mul2(mul2(mul2(Ts, Ts), sTs), X);
            den = fma2(bc2(k.sat), mul2(Ts, Vm), bc2(1.f));
        } else {
            const float2 T15 = mul2(Ts, sTs);
            num = mul2(T15, X);
            den = fma2(bc2(k.sat), Vm, T15);
        }
        return make_float2(ddiv<float>(num.x, den.x), ddiv<float>(num.y, den.y));
    }
    // upwind: F itself, blended with c_iso^3 from the donor cell of the normal flux
    const float2 nk = SP ? mul2(mul2(bc2(k.nk), mul2(Ts, Ts)), sTs) : bc2(k.nk);
    const float2 Fn = mul2(nk, X);
    const float2 Fmag = mul2(make_float2(fabsf(nk.x), fabsf(nk.y)), sqrt2(V2));
    const float2 Tq = make_float2(Fn.x >= 0.f ? TL.x : TR.x, Fn.y >= 0.f ? TL.y : TR.y);
    const float2 q = mul2(mul2(bc2(p.q0), Tq), sqrt2(Tq));
    const float2 den = add2(q, Fmag);
    return make_float2(ddiv<float>(q.x, den.x) * Fn.x, ddiv<float>(q.y, den.y) * Fn.y);
}

// --------------------------------------------------------------------------
// shared memory and copies

__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp16(unsigned d, const void* s)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(s));
}
__device__ __forceinline__ void st4(unsigned d, float v)
{
    asm volatile("st.shared.v4.f32 [%0], {%1, %1, %1, %1};\n" ::"r"(d), "f"(v));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ int pmod(int v, int n)
{
    int r = v % n;
    return r < 0 ? r + n : r;
}

__device__ __forceinline__ float2 lds2(const float* p) { return *reinterpret_cast<const float2*>(p); }

// --------------------------------------------------------------------------
// bulk copies on the TMA engine with mbarrier completion (sm_90+)

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_inval(unsigned bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(bar));
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity; false if it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity)
{
    for (int it = 0; it < (1 << 22); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it >= 16) __nanosleep(64);
    }
    return false;
}
// bytes (a multiple of 16) from global src to shared dst, both 16-byte
// aligned, completing on the mbarrier at bar
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

}  // namespace x2
}  // namespace rkl
