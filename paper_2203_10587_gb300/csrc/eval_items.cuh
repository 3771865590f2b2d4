// Per-item device functions of the polar AC-OPF model evaluation (ExaGO, arXiv 2203.10587,
// Sec. III, eqs. (7)-(10)), shared by the multi-kernel schedule (kernels.cu) and the persistent
// schedule (persist.cu).  Included by .cu files only.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace exago {

// What an item computes: g | h values, Jacobian values, Hessian values; W_GM compiles in the
// per-state generator mask (st_gmask), which a launch without one leaves out; W_PS compiles in
// phase-shifting transformers (the to end's own mutual admittances, when the net has them).
enum : int { W_G = 1, W_J = 2, W_H = 4, W_GM = 8, W_PS = 16 };

// Where state b's inputs and outputs live: row b of the batch arrays, or entry b of a gathered
// batch's state table.
__device__ __forceinline__ const double *st_x(const DevNet &N, const EvalReq &R, int b) {
    return R.tab ? R.tab[b].x : R.x + (size_t)b * N.n;
}
__device__ __forceinline__ const double *st_lam(const DevNet &N, const EvalReq &R, int b) {
    return R.tab ? R.tab[b].lam : R.lam + (size_t)b * N.m;
}
__device__ __forceinline__ const uint8_t *st_mask(const DevNet &N, const EvalReq &R, int b) {
    return R.tab ? R.tab[b].mask : R.mask ? R.mask + (size_t)b * N.nl : nullptr;
}
__device__ __forceinline__ const uint8_t *st_gmask(const DevNet &N, const EvalReq &R, int b) {
    return R.tab ? R.tab[b].gen_mask : R.gen_mask ? R.gen_mask + (size_t)b * N.ng : nullptr;
}
// Whether generator k of state b is in service (gm: st_gmask of the state).
__device__ __forceinline__ bool gen_on(const uint8_t *gm, int k) { return gm == nullptr || gm[k] != 0; }
__device__ __forceinline__ const double *st_pd(const DevNet &N, const EvalReq &R, int b) {
    return R.tab ? R.tab[b].pd_scale : R.pd_scale ? R.pd_scale + (size_t)b * N.nb : nullptr;
}
__device__ __forceinline__ double st_w(const EvalReq &R, int b) {
    const double *w = R.tab ? R.tab[b].obj_weight : R.obj_weight ? R.obj_weight + b : nullptr;
    return w ? *w : 1.0;
}
__device__ __forceinline__ double st_sigma(const EvalReq &R, int b) {
    return R.tab ? R.tab[b].sigma : R.sigma;
}
__device__ __forceinline__ double *st_f(const EvalReq &R, int b) { return R.tab ? R.tab[b].f : R.f + b; }
__device__ __forceinline__ double *st_grad(const DevNet &N, const EvalReq &R, int b) {
    return R.tab ? R.tab[b].grad : R.grad + (size_t)b * N.n;
}
__device__ __forceinline__ double *st_gh(const DevNet &N, const EvalReq &R, int b) {
    return R.tab ? R.tab[b].gh : R.gh + (size_t)b * N.m;
}
__device__ __forceinline__ double *st_jval(const DevNet &N, const EvalReq &R, int b) {
    return R.tab ? R.tab[b].jval : R.jval + (size_t)b * N.nnzJ;
}
__device__ __forceinline__ double *st_hval(const DevNet &N, const EvalReq &R, int b) {
    return R.tab ? R.tab[b].hval : R.hval + (size_t)b * N.nnzH;
}

// ---------------------------------------------------------------------------------------------
// sin and cos of the branch angle.  For |th| <= pi/4 -- every branch of a grid in normal
// operation -- minimax polynomials in z = th^2 (Remez exchange; the coefficients are written by
// paper_2203_10587_gb300/sincos_minimax.py, which states their derivation):
//   sin th = th + th^3 p(z),  cos th = 1 + z q(z),  p and q of degree 5,
// evaluated by Horner's rule with fused multiply-adds: 14 FP64 instructions for the pair, against
// about 28 for the library sincos, which is kept for larger angles.  Evaluated in this order the
// results are within 0.61 ulp (sin) and 1.17 ulp (cos) of the exact values (checked on the CPU
// with single-rounding fma).
// The library sincos for wide angles, kept out of line so that none of its instructions is
// scheduled ahead of the interval test and executed for every branch.
static __device__ __noinline__ void sincos_wide(double th, double *s, double *c) { sincos(th, s, c); }

__device__ __forceinline__ void branch_sincos(double th, double *s, double *c) {
    // |th| <= pi/4 by comparing bit patterns, in PTX so that it stays on the integer pipe
    int small;
    asm("{\n\t.reg .pred p;\n\t"
        "setp.le.u64 p, %1, 0x3FE921FB54442D18;\n\t"   // pi/4 rounded to double
        "selp.s32 %0, 1, 0, p;\n\t}"
        : "=r"(small)
        : "l"((unsigned long long)__double_as_longlong(th) & 0x7FFFFFFFFFFFFFFFull));
    if (small) {
        // SINCOS_COEFFS_BEGIN
        constexpr double p0 = -0x1.5555555555549p-3, p1 = 0x1.111111110f881p-7,
                         p2 = -0x1.a01a019c126c0p-13, p3 = 0x1.71de357875383p-19,
                         p4 = -0x1.ae5e66d592248p-26, p5 = 0x1.5d932f7c7cd31p-33;
        constexpr double q0 = -0x1.fffffffffff96p-2, q1 = 0x1.555555554f0abp-5,
                         q2 = -0x1.6c16c1640aabdp-10, q3 = 0x1.a019f81cb610fp-16,
                         q4 = -0x1.27df46099bb75p-22, q5 = 0x1.1b8b993bdb8c1p-29;
        // SINCOS_COEFFS_END
        const double z = th * th;
        const double u = fma(fma(fma(fma(fma(p5, z, p4), z, p3), z, p2), z, p1), z, p0);
        *s = fma(th * z, u, th);
        const double v = fma(fma(fma(fma(fma(q5, z, q4), z, q3), z, q2), z, q1), z, q0);
        *c = fma(v, z, 1.0);
    } else {
        sincos_wide(th, s, c);
    }
}

// The angle terms of both ends of branch l from s = sin th, c = cos th, th = Va_f - Va_t:
//   from end:  A_f = Gft c + Bft s,   C_f = Gft s - Bft c;
//   to end (angle -th):  A_t = Gtf c - Btf s,   C_t = -(Gtf s + Btf c).
// Without phase shift Gtf = Gft and Btf = Bft (G, Bm), and B c and B s serve both ends.  With PS
// and a net that has phase-shifting transformers (N.Gtf non-null) the to end reads its own pair.
template <bool PS>
__device__ __forceinline__ void angle_terms(const DevNet &N, int l, double G, double Bm, double s,
                                            double c, double *Af, double *Cf, double *At,
                                            double *Ct) {
    const double Bc = Bm * c, Bs = Bm * s;
    *Af = fma(G, c, Bs);
    *Cf = fma(G, s, -Bc);
    if (PS && N.Gtf) {
        const double Gt = __ldg(N.Gtf + l), Bt = __ldg(N.Btf + l);
        *At = fma(Gt, c, -(Bt * s));
        *Ct = -fma(Gt, s, Bt * c);
    } else {
        *At = fma(G, c, -Bs);
        *Ct = -fma(G, s, Bc);
    }
}

// 2 x, exactly, on the integer pipe (the FP64 pipe is the path's bottleneck): for a normal x
// whose double stays finite the exponent field goes up by one; zero and subnormals shift their
// magnitude bits left by one (the largest subnormals then become normal, as 2 x does); the
// largest binade goes to infinity; infinities and NaNs are returned unchanged.
__device__ __forceinline__ double twice(double x) {
    // written in PTX so that the compiler keeps it on the integer pipe
    double r;
    asm("{\n\t"
        ".reg .b64 b, s, m, e, t1, t2;\n\t"
        ".reg .pred p0, p1, p2;\n\t"
        "mov.b64 b, %1;\n\t"
        "and.b64 s, b, 0x8000000000000000;\n\t"
        "xor.b64 m, b, s;\n\t"
        "shr.u64 e, m, 52;\n\t"
        "shl.b64 t1, m, 1;\n\t"
        "or.b64 t1, t1, s;\n\t"                      // zero or subnormal: magnitude bits << 1
        "add.u64 t2, b, 0x0010000000000000;\n\t"     // normal: exponent + 1
        "setp.eq.u64 p0, e, 0;\n\t"
        "selp.b64 t2, t1, t2, p0;\n\t"
        "setp.eq.u64 p1, e, 0x7FE;\n\t"
        "or.b64 t1, s, 0x7FF0000000000000;\n\t"      // top binade: infinity
        "selp.b64 t2, t1, t2, p1;\n\t"
        "setp.eq.u64 p2, e, 0x7FF;\n\t"
        "selp.b64 t2, b, t2, p2;\n\t"                // infinity or NaN: unchanged
        "mov.b64 %0, t2;\n\t"
        "}"
        : "=d"(r)
        : "d"(x));
    return r;
}

// One end of a branch seen from its own bus u towards bus v:
//   P = Gss Vu^2 + Vu Vv A,  Q = -Bss Vu^2 + Vu Vv C,  A = G cos th_u + B sin th_u,
//   C = G sin th_u - B cos th_u,  th_u = Va_u - Va_v,
// and, since dA/dth = -C and dC/dth = A, its derivatives
//   dP/dth = -Vu Vv C,  dQ/dth = Vu Vv A,  dP/dVu = 2 Gss Vu + Vv A,  dQ/dVu = -2 Bss Vu + Vv C,
//   dP/dVv = Vu A,  dQ/dVv = Vu C.
struct End {
    double P, Q;
    double pa, pu, pv;   // dP / d(Va_u, Vm_u, Vm_v); dP/dVa_v = -pa
    double qa, qu, qv;   // dQ / d(Va_u, Vm_u, Vm_v)
};

// Gss2 = 2 Gss and Bss2 = 2 Bss (network tables); Vu2 = Vu^2 and VV = Vu Vv from the caller.
template <bool DERIV>
__device__ __forceinline__ End end_terms(double Gss, double Bss, double Gss2, double Bss2,
                                         double A, double C, double Vu, double Vv, double Vu2,
                                         double VV) {
    End e;
    e.qa = VV * A;                 //  Vu Vv A
    e.pa = -(VV * C);              // -Vu Vv C
    e.P = fma(Gss, Vu2, e.qa);
    e.Q = fma(-Bss, Vu2, -e.pa);
    if (DERIV) {
        e.pv = Vu * A;
        e.qv = Vu * C;
        e.pu = fma(Gss2, Vu, Vv * A);
        e.qu = fma(-Bss2, Vu, Vv * C);
    }
    return e;
}

// One end's Lagrangian Hessian block  lamP grad^2 P + lamQ grad^2 Q + mu grad^2 (P^2 + Q^2)  in
// (Va_u, Va_v, Vm_u, Vm_v), with wP = lamP + 2 mu P, wQ = lamQ + 2 mu Q, W1 = wP A + wQ C,
// W2 = wQ A - wP C and K = A^2 + C^2 = G^2 + B^2:
//   (Va_u,Va_u) = -(Va_u,Va_v) = (Va_v,Va_v) = 2 mu K (Vu Vv)^2 - Vu Vv W1;
//   (Va_u,Vm_u) = -(Va_v,Vm_u) = hau = 2 mu Vu Vv (A qu - C pu) + Vv W2;
//   (Va_u,Vm_v) = -(Va_v,Vm_v) = Vu W2;
//   (Vm_u,Vm_u) = huu = 2 mu (pu^2 + qu^2) + 2 Gss wP - 2 Bss wQ;
//   (Vm_u,Vm_v) = huv = 2 mu Vu (pu A + qu C) + W1;   (Vm_v,Vm_v) = 2 mu K Vu^2.
// The caller folds the two ends' blocks into the branch's values (branch_hess).
struct EndHess {
    double W1, W2, tK, hau, huu, huv;   // tK = 2 mu K
};

__device__ __forceinline__ EndHess end_hess(const End &e, double Gss2, double Bss2, double A,
                                            double C, double K, double Vu, double Vv,
                                            double lamP, double lamQ, double mu) {
    EndHess h;
    const double mu2 = twice(mu);
    const double wP = fma(mu2, e.P, lamP);
    const double wQ = fma(mu2, e.Q, lamQ);
    h.W1 = fma(wP, A, wQ * C);
    h.W2 = fma(wQ, A, -(wP * C));
    const double E = fma(A, e.qu, -(C * e.pu));
    const double F = fma(e.pu, A, e.qu * C);
    h.tK = mu2 * K;
    const double mu2Vu = mu2 * Vu;
    h.hau = Vv * fma(mu2Vu, E, h.W2);             // 2 mu Vu Vv E + Vv W2
    const double S = fma(e.pu, e.pu, e.qu * e.qu);
    h.huu = fma(mu2, S, fma(wP, Gss2, -(wQ * Bss2)));
    h.huv = fma(mu2Vu, F, h.W1);
    return h;
}

// The branch's Hessian values from its two ends' blocks:
//   (Va_f,Va_f) = haa = Vf Vt (Vf Vt (tK_f + tK_t) - (W1_f + W1_t));
//   (Vm_f, Va_f) = hau_f - Vt W2_t,  (Vm_t, Va_t) = hau_t - Vf W2_f;
//   (Vm_f, Vm_f) = huu_f + tK_t Vt^2,  (Vm_t, Vm_t) = huu_t + tK_f Vf^2,  (Vm_f, Vm_t) = huv_f + huv_t.
struct BranchHess {
    double haa, xf, xt, mff, mtt, mft;
};

__device__ __forceinline__ BranchHess branch_hess(const EndHess &hf, const EndHess &ht, double Vf,
                                                  double Vt, double Vf2, double Vt2, double VV) {
    BranchHess b;
    b.haa = VV * fma(VV, hf.tK + ht.tK, -(hf.W1 + ht.W1));
    b.xf = fma(-Vt, ht.W2, hf.hau);
    b.xt = fma(-Vf, hf.W2, ht.hau);
    b.mff = fma(ht.tK, Vt2, hf.huu);
    b.mtt = fma(hf.tK, Vf2, ht.huu);
    b.mft = hf.huv + ht.huv;
    return b;
}

// -x for a value that is only stored: the sign bit is flipped on the integer pipe, so that a
// negated store costs no FP64 instruction.
__device__ __forceinline__ double dneg(double v) {
    int hi = __double2hiint(v);
    const int lo = __double2loint(v);
    asm("xor.b32 %0, %0, 0x80000000;" : "+r"(hi));
    return __hiloint2double(hi, lo);
}

// h row of one end, |S|^2, and its four Jacobian entries in the row's ascending column order
// (Va_lo, Va_hi, Vm_lo, Vm_hi).
__device__ __forceinline__ void store_hrow(double *Jrow, const End &e, bool self_is_lo) {
    const double P2 = twice(e.P), Q2 = twice(e.Q);
    double da = fma(P2, e.pa, Q2 * e.qa);
    double du = fma(P2, e.pu, Q2 * e.qu);
    double dv = fma(P2, e.pv, Q2 * e.qv);
    const double nda = dneg(da);
    if (self_is_lo) {
        Jrow[0] = da; Jrow[1] = nda; Jrow[2] = du; Jrow[3] = dv;
    } else {
        Jrow[0] = nda; Jrow[1] = da; Jrow[2] = dv; Jrow[3] = du;
    }
}

// Stores the pair of components (c, c + 1) of a record, c even.  PS: doubles between a record's
// consecutive pairs -- 2 for a record of NCOMP consecutive doubles (16-byte aligned: records are
// 80 bytes), 64 for the lane-interleaved records of the warp-tiled schedule (a slot's pair p of
// 32 states is one 512-byte run, lane after lane).
template <int PS = 2>
__device__ __forceinline__ void put2(double *rec, int c, double a, double b) {
    *reinterpret_cast<double2 *>(rec + (c / 2) * PS) = make_double2(a, b);
}

// Where a branch item writes its two Jacobian h rows (four entries each) and its two h values
// instead of the state's J and g | h rows (the warp-tiled schedule's shared-memory staging); all
// null: the state's rows.
struct BranchOut {
    double *Jf = nullptr, *Jt = nullptr, *hf = nullptr, *ht = nullptr;
};

// One (state b, branch l) item.  scr is state b's record scratch ([nslot][NCOMP]), or with
// LW = 32 (warp-tiled schedule) a group of 32 states' records ([nslot][NCOMP / 2][32][2]) offset
// to the state's lane.  The branch writes its two h values and its two Jacobian h rows (four
// entries each), and the record of each end at the end's slot; the bus phase assembles
// everything else row by row.
template <int WANT, int LW = 1>
__device__ __forceinline__ void branch_item(const DevNet &N, const EvalReq &R, int b, int l,
                                            double *scr, const BranchOut &O = BranchOut{}) {
    constexpr bool WG = WANT & W_G, WJ = WANT & W_J, WH = WANT & W_H;
    constexpr bool DERIV = WG || WJ || WH;   // the bus balances come from derivative sums
    const int nb = N.nb, nl = N.nl;
    const int sf = __ldg(N.br_slot + l), sto = __ldg(N.br_slot + nl + l);
    const int fb = __ldg(N.f + l), tb = __ldg(N.t + l);
    if (!EXAGO_DCHECK(N, l >= 0 && l < nl && sf >= 0 && sf < N.chk_nslot && sto >= 0 &&
                             sto < N.chk_nslot && fb >= 0 && fb < nb && tb >= 0 && tb < nb))
        return;
    constexpr int PS = 2 * LW;                       // doubles between a record's pairs
    double *rf = scr + (size_t)sf * (NCOMP * LW);
    double *rt = scr + (size_t)sto * (NCOMP * LW);
    double *Jf = WJ ? (O.Jf ? O.Jf : st_jval(N, R, b) + N.nnzJg + 4 * (size_t)l) : nullptr;
    double *Jt = WJ ? (O.Jt ? O.Jt : st_jval(N, R, b) + N.nnzJg + 4 * (size_t)(nl + l)) : nullptr;
    double *ghb = R.gh ? st_gh(N, R, b) : nullptr;
    double *hrf = O.hf ? O.hf : ghb ? ghb + 2 * nb + l : nullptr;       // h rows of the ends
    double *hrt = O.ht ? O.ht : ghb ? ghb + 2 * nb + nl + l : nullptr;

    const uint8_t *mk = st_mask(N, R, b);
    const bool on = mk == nullptr || mk[l] != 0;
    if (!on) {   // out of service: every value of this branch is zero
#pragma unroll
        for (int e = 0; e < 2; e++) {
            double *r = e ? rt : rf;
            if (WG || WJ) { put2<PS>(r, SC_PA, 0.0, 0.0); put2<PS>(r, SC_PV, 0.0, 0.0); put2<PS>(r, SC_QU, 0.0, 0.0); }
            if (WH) { put2<PS>(r, SC_HAA, 0.0, 0.0); put2<PS>(r, SC_HUU, 0.0, 0.0); }
        }
        if (WG && ghb) { *hrf = 0.0; *hrt = 0.0; }
        if (WJ)
            for (int k = 0; k < 4; k++) { Jf[k] = 0.0; Jt[k] = 0.0; }
        return;
    }

    const double *xb = st_x(N, R, b);
    const double Vaf = __ldg(xb + fb), Vat = __ldg(xb + tb);
    const double Vf = __ldg(xb + nb + fb), Vt = __ldg(xb + nb + tb);
    const double G = __ldg(N.Gft + l), Bm = __ldg(N.Bft + l);
    const double Gff = __ldg(N.Gff + l), Bff = __ldg(N.Bff + l);
    const double Gtt = __ldg(N.Gtt + l), Btt = __ldg(N.Btt + l);
    const double Gff2 = __ldg(N.Gff2 + l), Bff2 = __ldg(N.Bff2 + l);
    const double Gtt2 = __ldg(N.Gtt2 + l), Btt2 = __ldg(N.Btt2 + l);

    double s, c;
    branch_sincos(Vaf - Vat, &s, &c);
    double Af, Cf, At, Ct;    // from end, th = Va_f - Va_t; to end, th = Va_t - Va_f
    angle_terms<(WANT & W_PS) != 0>(N, l, G, Bm, s, c, &Af, &Cf, &At, &Ct);
    const double VV = Vf * Vt, Vf2 = Vf * Vf, Vt2 = Vt * Vt;

    // One end at a time, stored as soon as it is computed, so that fewer values are live at once
    // (the compiler would otherwise recompute products to save registers).
    const double *lb = WH ? st_lam(N, R, b) : nullptr;
    const double K = WH ? __ldg(N.Kft + l) : 0.0;    // A^2 + C^2 = G^2 + B^2 at both ends
    EndHess hf{}, ht{};
    {
        const End ef = end_terms<DERIV>(Gff, Bff, Gff2, Bff2, Af, Cf, Vf, Vt, Vf2, VV);
        if (WG && ghb) *hrf = fma(ef.P, ef.P, ef.Q * ef.Q);
        if (WG || WJ) {
            put2<PS>(rf, SC_PA, ef.pa, ef.pu); put2<PS>(rf, SC_PV, ef.pv, ef.qa); put2<PS>(rf, SC_QU, ef.qu, ef.qv);
        }
        if (WJ) store_hrow(Jf, ef, fb < tb);
        if (WH)
            hf = end_hess(ef, Gff2, Bff2, Af, Cf, K, Vf, Vt, __ldg(lb + fb), __ldg(lb + nb + fb),
                          __ldg(lb + 2 * nb + l));
    }
    {
        const End et = end_terms<DERIV>(Gtt, Btt, Gtt2, Btt2, At, Ct, Vt, Vf, Vt2, VV);
        if (WG && ghb) *hrt = fma(et.P, et.P, et.Q * et.Q);
        if (WG || WJ) {
            put2<PS>(rt, SC_PA, et.pa, et.pu); put2<PS>(rt, SC_PV, et.pv, et.qa); put2<PS>(rt, SC_QU, et.qu, et.qv);
        }
        if (WJ) store_hrow(Jt, et, tb < fb);
        if (WH)
            ht = end_hess(et, Gtt2, Btt2, At, Ct, K, Vt, Vf, __ldg(lb + tb), __ldg(lb + nb + tb),
                          __ldg(lb + 2 * nb + nl + l));
    }
    if (WH) {
        const BranchHess h = branch_hess(hf, ht, Vf, Vt, Vf2, Vt2, VV);
        put2<PS>(rf, SC_HAA, h.haa, h.xf);                 // (Va_f,Va_f), (Vm_f, Va_f)
        put2<PS>(rt, SC_HAA, h.haa, h.xt);                 // (Va_t,Va_t), (Vm_t, Va_t)
        put2<PS>(rf, SC_HUU, h.mff, h.mft);
        put2<PS>(rt, SC_HUU, h.mtt, h.mft);
    }
}

// Gradient entry of generator k's active power: w (2 c2 base^2 Pg + c1 base), with the network
// constants c2g = 2 c2 base^2 and c1g = c1 base.
template <bool GM>
__device__ __forceinline__ double grad_pg(const DevNet &N, const EvalReq &R, int b, int k) {
    if constexpr (GM) {
        if (!gen_on(st_gmask(N, R, b), k)) return 0.0;    // generator out of service
    }
    const double w = st_w(R, b);
    const double Pg = __ldg(st_x(N, R, b) + 2 * N.nb + k);
    return w * fma(__ldg(N.c2g + k), Pg, __ldg(N.c1g + k));
}

// Where one bus writes its Jacobian rows P_i, Q_i and Hessian rows Va_i, Vm_i (global memory, or
// a shared-memory staging copy of the tile's row segments).
struct BusRows {
    double *JP, *JQ, *HA, *HM;
};

__device__ __forceinline__ double2 ld2(const double *p) {
    return __ldcg(reinterpret_cast<const double2 *>(p));
}

// The values of one branch-end record that a request needs.
struct Rec {
    double pa, pu, pv, qa, qu, qv, haa, hua, huu, huv;
};

// A record pair from shared memory (SMEM) or through L2 (records other CTAs wrote this launch).
template <bool SMEM>
__device__ __forceinline__ double2 rec2(const double *p) {
    if (SMEM) return *reinterpret_cast<const double2 *>(p);
    return ld2(p);
}

// PS: doubles between the record's pairs (put2).
template <int WANT, bool SMEM, int PS = 2>
__device__ __forceinline__ Rec load_rec(const double *rec) {
    Rec r{};
    if (WANT & (W_G | W_J)) {
        const double2 a = rec2<SMEM>(rec + SC_PA / 2 * PS), v = rec2<SMEM>(rec + SC_PV / 2 * PS);
        const double2 u = rec2<SMEM>(rec + SC_QU / 2 * PS);
        r.pa = a.x; r.pu = a.y; r.pv = v.x; r.qa = v.y; r.qu = u.x; r.qv = u.y;
    }
    if (WANT & W_H) {
        const double2 h1 = rec2<SMEM>(rec + SC_HAA / 2 * PS), h2 = rec2<SMEM>(rec + SC_HUU / 2 * PS);
        r.haa = h1.x; r.hua = h1.y; r.huu = h2.x; r.huv = h2.y;
    }
    return r;
}

// Diagonal sums of a bus: dP/dVa_u, dP/dVm_u, dQ/dVa_u, dQ/dVm_u, H diagonal terms.
template <int WANT>
__device__ __forceinline__ void add_diag(Rec &d, const Rec &r) {
    if (WANT & (W_G | W_J)) { d.pa += r.pa; d.pu += r.pu; d.qa += r.qa; d.qu += r.qu; }
    if (WANT & W_H) { d.haa += r.haa; d.hua += r.hua; d.huu += r.huu; }
}

// Off-diagonal entries towards one neighbour, summed over parallel branches.
template <int WANT>
__device__ __forceinline__ void add_group(Rec &o, const Rec &r) {
    if (WANT & W_J) { o.pa += r.pa; o.pv += r.pv; o.qa += r.qa; o.qv += r.qv; }
    if (WANT & W_H) { o.haa += r.haa; o.hua += r.hua; o.huv += r.huv; }
}

// The rest of one (state b, bus i) item once D holds the sums of the bus's branch-end records
// (the diagonal derivative and Hessian terms):
//   g:  P_i and Q_i balances (injections, load and generators).  The injections are
//       homogeneous of degree 2 in the voltage magnitudes, so (Euler) 2 P_i = Vm_i dP_i/dVm_i +
//       sum over the ends of Vm_v dP/dVm_v, and Vm_v dP/dVm_v = Vu Vv A is the end's dQ/dVa_u;
//       likewise 2 Q_i = Vm_i dQ_i/dVm_i - sum of dP/dVa_u.  An out-of-service end's record is
//       zero, so no end's injection needs summing on its own;
//   J:  the diagonal entries of rows P_i and Q_i (plus the shunt term) and -1 for each generator;
//   H:  the diagonals of rows Va_i and Vm_i (plus the shunt term) and the cost Hessian of the
//       bus's generators.
// A generator out of service (st_gmask) injects nothing and its -1 and cost Hessian entries are 0.
template <int WANT>
__device__ __forceinline__ void bus_tail(const DevNet &N, const EvalReq &R, int b, int i,
                                         const Rec &D, const BusRows &W) {
    constexpr bool WG = WANT & W_G, WJ = WANT & W_J, WH = WANT & W_H, GM = WANT & W_GM;
    const int nb = N.nb;
    const int g0 = __ldg(N.gen_ptr + i), g1 = __ldg(N.gen_ptr + i + 1);
    if (!EXAGO_DCHECK(N, g0 >= 0 && g0 <= g1 && g1 <= N.ng)) return;
    const double *xb = st_x(N, R, b);
    const double Vm = __ldg(xb + nb + i);
    const double Gs = __ldg(N.Gs + i), Bs = __ldg(N.Bs + i);
    const int k = __ldg(N.bus_k + i), nlow = __ldg(N.bus_nlow + i);
    double *JP = W.JP, *JQ = W.JQ, *HA = W.HA, *HM = W.HM;
    const double dPa = D.pa, dPu = D.pu, dQa = D.qa, dQu = D.qu;
    const double dAA = D.haa, dUA = D.hua, dUU = D.huu;
    // dP_i/dVm_i and dQ_i/dVm_i, with the shunt terms
    const double tV = twice(Vm);
    const double JPu = fma(Gs, tV, dPu), JQu = fma(-Bs, tV, dQu);
    [[maybe_unused]] const uint8_t *gm = nullptr;
    if constexpr (GM) gm = g1 > g0 ? st_gmask(N, R, b) : nullptr;

    if (WG && R.gh) {
        double Pd = __ldg(N.Pd + i), Qd = __ldg(N.Qd + i);
        const double *pds = st_pd(N, R, b);
        if (pds) {                                            // load scenarios
            const double sc = __ldg(pds + i);
            Pd *= sc;
            Qd *= sc;
        }
        double gP = fma(0.5, fma(Vm, JPu, dQa), Pd);
        double gQ = fma(0.5, fma(Vm, JQu, -dPa), Qd);
        for (int q = g0; q < g1; q++) {
            const int g = __ldg(N.gen_ord + q);
            if constexpr (GM) {
                if (!gen_on(gm, g)) continue;
            }
            gP -= __ldg(xb + 2 * nb + g);
            gQ -= __ldg(xb + 2 * nb + N.ng + g);
        }
        double *ghb = st_gh(N, R, b);
        ghb[i] = gP;
        ghb[nb + i] = gQ;
    }
    if (WJ) {
        JP[nlow] = dPa; JP[k + nlow] = JPu;
        JQ[nlow] = dQa; JQ[k + nlow] = JQu;
        for (int q = 0; q < g1 - g0; q++) {
            if constexpr (GM) {
                const double v = gen_on(gm, gm ? __ldg(N.gen_ord + g0 + q) : 0) ? -1.0 : 0.0;
                JP[2 * k + q] = v;
                JQ[2 * k + q] = v;
            } else {
                JP[2 * k + q] = -1.0;
                JQ[2 * k + q] = -1.0;
            }
        }
    }
    if (WH) {
        const double *lb = st_lam(N, R, b);
        const double lP = __ldg(lb + i), lQ = __ldg(lb + nb + i);
        HA[nlow] = dAA;                                       // (Va_i, Va_i): last of row Va_i
        HM[nlow] = dUA;                                       // (Vm_i, Va_i)
        HM[k + nlow] = dUU + fma(lP, twice(Gs), -(lQ * twice(Bs)));   // (Vm_i, Vm_i): last
        if (g1 > g0) {
            const double sw = st_sigma(R, b) * st_w(R, b);
            double *Hb = st_hval(N, R, b) + N.hpg;
            for (int q = g0; q < g1; q++) {
                const int g = __ldg(N.gen_ord + q);
                if constexpr (GM) Hb[g] = gen_on(gm, g) ? sw * __ldg(N.c2g + g) : 0.0;
                else Hb[g] = sw * __ldg(N.c2g + g);
            }
        }
    }
}

// One (state b, bus i) item.  Walks the bus's slots, which come in ascending order of the other
// bus (parallel branches adjacent), reads each slot's branch-end record, writes the bus's
// off-diagonal row entries (a neighbour's J entry is its branch end's dP/dVa_v = -dP/dVa_u and
// dP/dVm_v; its H entries the end's Hessian values), sums the diagonal terms and finishes with
// bus_tail.  Records come from the tile's shared-memory copy, or through L2 (ld.cg): in the
// persistent schedule other CTAs wrote them during the launch.  recs + (s - sbase) * NCOMP is slot
// s's record: the tile's shared-memory copy (SMEM) or state b's scratch in global memory
// (sbase = 0).  LW = 32: the warp-tiled schedule's lane-interleaved records (branch_item), recs
// offset to the state's lane; every lane of a warp then walks the same bus.
template <int WANT, bool SMEM, int LW = 1>
__device__ __forceinline__ void bus_item(const DevNet &N, const EvalReq &R, int b, int i,
                                         const double *recs, int sbase, const BusRows &W) {
    constexpr bool WJ = WANT & W_J, WH = WANT & W_H;
    const int s0 = __ldg(N.slot_ptr + i), s1 = __ldg(N.slot_ptr + i + 1);
    const int k = __ldg(N.bus_k + i), nlow = __ldg(N.bus_nlow + i);
    double *JP = W.JP, *JQ = W.JQ, *HA = W.HA, *HM = W.HM;
    if (!EXAGO_DCHECK(N, i >= 0 && i < N.nb && s0 >= 0 && s0 <= s1 && s1 <= N.chk_nslot &&
                             nlow >= 0 && nlow < k && s1 - s0 >= k - 1))
        return;

    // The first record of the bus initialises the diagonal sums and the first neighbour's entries;
    // every later record adds to the diagonal sums and starts (or, for a parallel branch, adds to)
    // its neighbour's entries.  Warps hold buses of similar degree (bus_perm), so the loop below
    // runs nearly converged: the FP64 pipe is charged per warp instruction, not per active lane.
    Rec D{};
    int pos = 0;                                                    // column among cols_i
    auto emit = [&](int j, const Rec &o) {
        if (pos == nlow) pos++;   // the diagonal column sits between the lower and upper neighbours
        if (WJ) {
            JP[pos] = dneg(o.pa); JP[k + pos] = o.pv;
            JQ[pos] = dneg(o.qa); JQ[k + pos] = o.qv;
        }
        if (WH) {
            HM[pos] = dneg(o.hua);                            // (Vm_i, Va_j)
            if (j < i) {
                HA[pos] = dneg(o.haa);                        // (Va_i, Va_j)
                HM[k + pos] = o.huv;                          // (Vm_i, Vm_j)
            }
        }
        pos++;
    };
    auto rec_of = [&](int s) { return recs + (size_t)(s - sbase) * (NCOMP * LW); };
    int s = s0;
    if (s < s1) {
        int j = __ldg(N.slot_nbr + s);
        Rec o = load_rec<WANT, SMEM, 2 * LW>(rec_of(s));
        D = o;
        for (;;) {
            s++;
            int jn = s < s1 ? __ldg(N.slot_nbr + s) : -1;
            while (jn == j) {                                 // parallel branch to the same bus
                const Rec p = load_rec<WANT, SMEM, 2 * LW>(rec_of(s));
                add_group<WANT>(o, p);
                add_diag<WANT>(D, p);
                s++;
                jn = s < s1 ? __ldg(N.slot_nbr + s) : -1;
            }
            emit(j, o);
            if (s >= s1) break;
            j = jn;
            o = load_rec<WANT, SMEM, 2 * LW>(rec_of(s));
            add_diag<WANT>(D, o);
        }
    }
    bus_tail<WANT>(N, R, b, i, D, W);
}

// Start of bus i's row in one of the four row blocks, or the block's end for i = nb.
__device__ __forceinline__ int row_start(const int *starts, int i, int nb, int end) {
    return i < nb ? __ldg(starts + i) : end;
}

// The threads that share one bus tile: a whole block of 64, 128 or 256 threads.
struct BlockGroup {
    static __device__ __forceinline__ int rank() { return threadIdx.x; }
    static __device__ __forceinline__ int size() { return blockDim.x; }
    static __device__ __forceinline__ void sync() { __syncthreads(); }
};

// Where a bus tile's rows go: the start of the tile's segment in each of the four row blocks
// (shared-memory staging or global memory) and the blocks' first positions p0, q0, a0, m0.
struct TileRows {
    double *P, *Q, *A, *M;
    int p0, q0, a0, m0;
    template <int WANT>
    __device__ __forceinline__ BusRows of(const DevNet &N, int i) const {
        BusRows W{};
        if (WANT & W_J) {
            W.JP = P + (__ldg(N.bus_jP + i) - p0);
            W.JQ = Q + (__ldg(N.bus_jQ + i) - q0);
        }
        if (WANT & W_H) {
            W.HA = A + (__ldg(N.bus_hA + i) - a0);
            W.HM = M + (__ldg(N.bus_hM + i) - m0);
        }
        return W;
    }
};

// Slot-parallel first phase of a bus tile, for slot s of bus i = slot_bus[s]: reads the slot's
// record (consecutive slots are consecutive records, so a warp's loads are coalesced), keeps its
// diagonal components in dg[0 .. kDiagComps) of shared memory, and -- if the slot leads its
// neighbour group -- sums the group's later parallel branches in slot order and writes the
// neighbour's row entries, exactly as bus_item does.
template <int WANT>
__device__ __forceinline__ void slot_item(const DevNet &N, int s, const double *scr, double *dg,
                                          const TileRows &T) {
    constexpr bool WG = WANT & W_G, WJ = WANT & W_J, WH = WANT & W_H;
    if (!EXAGO_DCHECK(N, s >= 0 && s < N.chk_nslot)) return;
    Rec o = load_rec<WANT, false>(scr + (size_t)s * NCOMP);
    if (WG || WJ) { dg[0] = o.pa; dg[1] = o.pu; dg[2] = o.qa; dg[3] = o.qu; }
    if (WH) { dg[4] = o.haa; dg[5] = o.hua; dg[6] = o.huu; }
    const int pos = __ldg(N.slot_pos + s);
    if (!(WJ || WH) || pos < 0) return;
    const int i = __ldg(N.slot_bus + s), j = __ldg(N.slot_nbr + s);
    const int e = __ldg(N.slot_ptr + i + 1);
    for (int q = s + 1; q < e && __ldg(N.slot_nbr + q) == j; q++)
        add_group<WANT>(o, load_rec<WANT, false>(scr + (size_t)q * NCOMP));
    const int k = __ldg(N.bus_k + i);
    const BusRows W = T.template of<WANT>(N, i);
    if (WJ) {
        W.JP[pos] = dneg(o.pa); W.JP[k + pos] = o.pv;
        W.JQ[pos] = dneg(o.qa); W.JQ[k + pos] = o.qv;
    }
    if (WH) {
        W.HM[pos] = dneg(o.hua);                              // (Vm_i, Va_j)
        if (j < i) {
            W.HA[pos] = dneg(o.haa);                          // (Va_i, Va_j)
            W.HM[k + pos] = o.huv;                            // (Vm_i, Vm_j)
        }
    }
}

// Second phase for bus i: the diagonal sums over its slots' components in slot order (the same
// additions as bus_item), then bus_tail.
template <int WANT>
__device__ __forceinline__ void bus_sums(const DevNet &N, const EvalReq &R, int b, int i, int S0,
                                         const double *dgs, const BusRows &W) {
    constexpr bool WG = WANT & W_G, WJ = WANT & W_J, WH = WANT & W_H;
    const int s0 = __ldg(N.slot_ptr + i), s1 = __ldg(N.slot_ptr + i + 1);
    Rec D{};
    for (int s = s0; s < s1; s++) {
        const double *d = dgs + (size_t)(s - S0) * kDiagComps;
        Rec r{};
        if (WG || WJ) { r.pa = d[0]; r.pu = d[1]; r.qa = d[2]; r.qu = d[3]; }
        if (WH) { r.haa = d[4]; r.hua = d[5]; r.huu = d[6]; }
        if (s == s0) D = r;
        else add_diag<WANT>(D, r);
    }
    bus_tail<WANT>(N, R, b, i, D, W);
}

// Bulk copy of a bus tile's records into shared memory (the persistent kernel): one TMA bulk
// copy (cp.async.bulk) whose completion an mbarrier of the CTA counts.  mbar: the barrier
// (initialised with an arrival count of 1); a wait gives up after spin_limit polls.  The parity
// of the barrier's next completion is kept by every thread of the CTA (bus_tile's `phase`).
struct BulkCtx {
    unsigned long long *mbar;
    long long spin_limit;
};

// Thread 0: the tile's records [src, src + bytes) -> dst (shared memory), both 16-byte aligned
// and bytes a multiple of 16.  The group's earlier shared-memory accesses of dst are ordered
// before the copy by the caller's barrier and the proxy fence here; the records were written by
// other CTAs and acquired through the tile's wait.
__device__ __forceinline__ void bulk_records(double *dst, const double *src, unsigned bytes,
                                             unsigned long long *mbar) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const unsigned m = (unsigned)__cvta_generic_to_shared(mbar);
    asm volatile("fence.proxy.async;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(m), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(d), "l"(src), "r"(bytes), "r"(m)
                 : "memory");
}

// Every thread: waits for the barrier's completion of the given parity; false (and a timeout
// code in the status word) after `limit` polls.
__device__ __forceinline__ bool bulk_wait(unsigned long long *mbar, unsigned parity,
                                          long long limit, int *status) {
    const unsigned m = (unsigned)__cvta_generic_to_shared(mbar);
    for (long long it = 0;; it++) {
        unsigned done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(m), "r"(parity)
                     : "memory");
        if (done) return true;
        if (it >= limit) {
            if (status) *(volatile int *)status = 3;   // the records' bulk copy did not complete
            return false;
        }
    }
}

// The bus items of buses [i0, i0 + G::size()) of state b, by the whole group (i0 a multiple of
// the group size), with `stage` = cap doubles of shared memory.  The tile's slots are one
// contiguous range [S0, S1), and its rows are four contiguous segments.
//   * With R.stage_recs == 1, and when the slots' diagonal components fit, the tile runs
//     slot-parallel: every thread takes slots (slot_item), then every thread sums its bus's
//     components from shared memory (bus_sums).
//   * With R.stage_recs == 2, a bulk context (the persistent kernel) and when the tile's records
//     fit, one bulk copy brings them into shared memory and every thread walks its own bus's
//     slots there (bus_item).
//   * Otherwise every thread walks its own bus's slots, reading the records through L2
//     (bus_item).
// When the row segments fit (after the components, if used), every row entry is written to
// shared memory and the group copies the four segments out with coalesced stores; otherwise
// the rows go straight to global memory.  Contains G::sync(): call from every thread.
template <int WANT, class G>
__device__ __forceinline__ void bus_tile(const DevNet &N, const EvalReq &R, int b, int i0,
                                         const double *scr, double *stage, int cap,
                                         const BulkCtx *bk = nullptr, unsigned *phase = nullptr) {
    constexpr bool WJ = WANT & W_J, WH = WANT & W_H;
    const int nb = N.nb, r = G::rank(), sz = G::size();
    int i1 = i0 + sz;
    if (i1 > nb) i1 = nb;
    // thread -> bus through the tile size's degree-sorted permutation (it maps every tile onto
    // itself)
    const int *perm = N.bus_perm + (size_t)stage_index(sz) * nb;
    const int i = i0 + r < i1 ? __ldg(perm + i0 + r) : nb;
    const int S0 = __ldg(N.slot_ptr + i0), S1 = __ldg(N.slot_ptr + i1);
    const int p0 = row_start(N.bus_jP, i0, nb, N.jP_end), p1 = row_start(N.bus_jP, i1, nb, N.jP_end);
    const int q0 = row_start(N.bus_jQ, i0, nb, N.jQ_end);
    const int a0 = row_start(N.bus_hA, i0, nb, N.hA_end), a1 = row_start(N.bus_hA, i1, nb, N.hA_end);
    const int m0 = row_start(N.bus_hM, i0, nb, N.hM_end), m1 = row_start(N.bus_hM, i1, nb, N.hM_end);
    const int LP = WJ ? p1 - p0 : 0, LA = WH ? a1 - a0 : 0, LM = WH ? m1 - m0 : 0;
    const int LROWS = 2 * LP + LA + LM;
    // slot-parallel whenever the components fit, or the records in bulk whenever they fit; the
    // rows are staged after them when they fit too
    const bool slotpar = R.stage_recs == 1 && kDiagComps * (S1 - S0) <= cap;
    const bool bulk = bk != nullptr && phase != nullptr && R.stage_recs == 2 && S1 > S0 &&
                      NCOMP * (S1 - S0) <= cap;
    const int LD = slotpar ? kDiagComps * (S1 - S0) : bulk ? NCOMP * (S1 - S0) : 0;
    const bool staged = (WJ || WH) && LD + LROWS <= cap;
    double *Jb = WJ ? st_jval(N, R, b) : nullptr;
    double *Hb = WH ? st_hval(N, R, b) : nullptr;
    double *rows = stage + LD;
    TileRows T{};
    T.p0 = p0; T.q0 = q0; T.a0 = a0; T.m0 = m0;
    if (staged) {
        T.P = rows; T.Q = rows + LP; T.A = rows + 2 * LP; T.M = rows + 2 * LP + LA;
    } else {
        if (WJ) { T.P = Jb + p0; T.Q = Jb + q0; }
        if (WH) { T.A = Hb + a0; T.M = Hb + m0; }
    }
    if (slotpar) {
        for (int s = S0 + r; s < S1; s += sz)
            slot_item<WANT>(N, s, scr, stage + (size_t)(s - S0) * kDiagComps, T);
        G::sync();
        if (i < i1) bus_sums<WANT>(N, R, b, i, S0, stage, T.template of<WANT>(N, i));
    } else if (bulk) {
        if (r == 0)
            bulk_records(stage, scr + (size_t)S0 * NCOMP, (unsigned)(LD * sizeof(double)), bk->mbar);
        const bool ok = bulk_wait(bk->mbar, *phase, bk->spin_limit, N.status);
        *phase ^= 1u;
        if (i < i1 && ok) bus_item<WANT, true>(N, R, b, i, stage, S0, T.template of<WANT>(N, i));
    } else if (i < i1) {
        bus_item<WANT, false>(N, R, b, i, scr, 0, T.template of<WANT>(N, i));
    }
    if (staged) {
        G::sync();
        for (int e = r; e < LP; e += sz) {
            Jb[p0 + e] = rows[e];
            Jb[q0 + e] = rows[LP + e];
        }
        for (int e = r; e < LA; e += sz) Hb[a0 + e] = rows[2 * LP + e];
        for (int e = r; e < LM; e += sz) Hb[m0 + e] = rows[2 * LP + LA + e];
        G::sync();
    } else if (slotpar || bulk) {
        G::sync();   // the next tile may overwrite the components or records
    }
}

// Gradient entries owned by bus i: Va_i and Vm_i (zero) and, for each generator at i, Pg and Qg.
template <bool GM>
__device__ __forceinline__ void grad_bus(const DevNet &N, const EvalReq &R, int b, int i) {
    double *gb = st_grad(N, R, b);
    gb[i] = 0.0;
    gb[N.nb + i] = 0.0;
    const int g0 = __ldg(N.gen_ptr + i), g1 = __ldg(N.gen_ptr + i + 1);
    for (int s = g0; s < g1; s++) {
        const int k = __ldg(N.gen_ord + s);
        gb[2 * N.nb + k] = grad_pg<GM>(N, R, b, k);
        gb[2 * N.nb + N.ng + k] = 0.0;
    }
}

// Objective of state b, f = w sum_k (c2 MW^2 + c1 MW + c0), MW = base Pg, by the whole block.
// Virtual lane v < 256 sums generators v, v+256, ... in order; the 256 partials are combined by
// a fixed pairwise tree.  The result is the same for every block size.  part: 256 doubles of
// shared memory.
constexpr int OBJ_LANES = kObjLanes;
// NT: the block's threads (a divisor of OBJ_LANES).
template <bool GM, int NT>
__device__ __forceinline__ void obj_block(const DevNet &N, const EvalReq &R, int b, double *part) {
    static_assert(NT >= 32 && OBJ_LANES % NT == 0, "block size");
    constexpr int LPT = OBJ_LANES / NT;   // virtual lanes per thread
    const double *Pg = st_x(N, R, b) + 2 * N.nb;
    [[maybe_unused]] const uint8_t *gm = nullptr;
    if constexpr (GM) gm = st_gmask(N, R, b);
    // Thread r holds lanes r, r + NT, ...  Each step loads the next two generators of all of them
    // before adding, so that one thread has many loads in flight; every lane still adds its
    // generators in increasing order.  A missing generator (past ng, or out of service) adds
    // +0.0, which leaves the sum unchanged: it starts at +0.0, so it is never -0.0.
    double acc[LPT];
#pragma unroll
    for (int j = 0; j < LPT; j++) acc[j] = 0.0;
    auto term = [&](int v, int r) -> double {
        const int k = v + r * OBJ_LANES;
        if (k >= N.ng) return 0.0;
        if constexpr (GM) {
            if (!gen_on(gm, k)) return 0.0;                   // generator out of service
        }
        const double MW = N.baseMVA * __ldg(Pg + k);
        return fma(fma(__ldg(N.c2 + k), MW, __ldg(N.c1 + k)), MW, __ldg(N.c0 + k));
    };
    const int rounds = (N.ng + OBJ_LANES - 1) / OBJ_LANES;
    for (int r = 0; r < rounds; r += 2) {
        double t0[LPT], t1[LPT];
#pragma unroll
        for (int j = 0; j < LPT; j++) {
            t0[j] = term(threadIdx.x + j * NT, r);
            t1[j] = term(threadIdx.x + j * NT, r + 1);
        }
#pragma unroll
        for (int j = 0; j < LPT; j++) acc[j] = (acc[j] + t0[j]) + t1[j];
    }
#pragma unroll
    for (int j = 0; j < LPT; j++) part[threadIdx.x + j * NT] = acc[j];
    __syncthreads();
    for (int w = OBJ_LANES / 2; w > 0; w >>= 1) {
        for (int v = threadIdx.x; v < w; v += NT) part[v] += part[v + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *st_f(R, b) = st_w(R, b) * part[0];
    __syncthreads();
}


// The objective of state b split over several CTAs (the persistent schedule): lanes
// [q NT, (q + 1) NT) of obj_block's 256 virtual lanes, one per thread, each summing its generators
// in increasing order exactly as obj_block does, into partials[v] (global memory).
template <bool GM, int NT>
__device__ __forceinline__ void obj_lanes(const DevNet &N, const EvalReq &R, int b, int q,
                                          double *partials) {
    const double *Pg = st_x(N, R, b) + 2 * N.nb;
    [[maybe_unused]] const uint8_t *gm = nullptr;
    if constexpr (GM) gm = st_gmask(N, R, b);
    const int v = q * NT + threadIdx.x;
    auto term = [&](int k) -> double {
        if (k >= N.ng) return 0.0;
        if constexpr (GM) {
            if (!gen_on(gm, k)) return 0.0;                   // generator out of service
        }
        const double MW = N.baseMVA * __ldg(Pg + k);
        return fma(fma(__ldg(N.c2 + k), MW, __ldg(N.c1 + k)), MW, __ldg(N.c0 + k));
    };
    // four generators' loads in flight before their terms are added in order (+0.0 for a missing
    // one leaves the sum unchanged, as in obj_block)
    double acc = 0.0;
    for (int k = v; k < N.ng; k += 4 * OBJ_LANES) {
        const double t0 = term(k), t1 = term(k + OBJ_LANES), t2 = term(k + 2 * OBJ_LANES),
                     t3 = term(k + 3 * OBJ_LANES);
        acc = (((acc + t0) + t1) + t2) + t3;
    }
    partials[v] = acc;
}

// obj_block's fixed pairwise tree over the 256 partials, by one warp (lanes 0..31 of the
// calling warp): levels 128, 64 and 32 in registers (lane l holds lanes l + 32 j), then 16 .. 1
// by shuffles, each level adding part[v + w] to part[v] for v < w as obj_block does, so the
// result is bitwise obj_block's.  Writes f[b].  partials were written by other CTAs of the launch
// (read through L2).
__device__ __forceinline__ void obj_tree_warp(const EvalReq &R, int b, const double *partials) {
    const int l = threadIdx.x & 31;
    double p[8];
#pragma unroll
    for (int j = 0; j < 8; j++) p[j] = __ldcg(partials + l + 32 * j);
#pragma unroll
    for (int j = 0; j < 4; j++) p[j] += p[j + 4];
    p[0] += p[2];
    p[1] += p[3];
    p[0] += p[1];
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const double o = __shfl_down_sync(0xffffffffu, p[0], w);
        if (l < w) p[0] += o;
    }
    if (l == 0) *st_f(R, b) = st_w(R, b) * p[0];
}

// Records an event on the launching stream before a kernel when profiling.
static inline void mark(ProfileHook *hk, cudaStream_t st, const char *name) {
    if (!hk || hk->n >= ProfileHook::MAX - 1) return;
    cudaEventRecord(hk->ev[hk->n], st);
    hk->name[hk->n] = name;
    hk->n++;
}

}  // namespace exago
