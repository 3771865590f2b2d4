// Per-item device functions of the polar AC-OPF model evaluation (ExaGO, arXiv 2203.10587,
// Sec. III, eqs. (7)-(10)), shared by the multi-kernel schedule (kernels.cu) and the persistent
// schedule (persist.cu).  Included by .cu files only.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace exago {

enum : int { W_G = 1, W_J = 2, W_H = 4 };

// ---------------------------------------------------------------------------------------------
// sin and cos of the branch angle.  For |th| <= pi/4 -- every branch of a grid in normal
// operation -- their Taylor series are summed by Horner's rule in z = th^2, truncated after th^15
// (sin) and th^16 (cos): on that interval the first omitted terms are below 5e-17 and 2e-18, under
// half an ulp of the results.  That is 17 FP64 instructions, against about 28 for the library
// sincos (measured throughput), which is kept for larger angles.  The interval test compares the
// bit pattern of |th| with that of pi/4 on the integer pipe.
__device__ __forceinline__ void branch_sincos(double th, double *s, double *c) {
    const unsigned long long PI4_BITS = 0x3FE921FB54442D18ull;   // pi/4 rounded to double
    if ((__double_as_longlong(th) & 0x7FFFFFFFFFFFFFFFull) <= PI4_BITS) {
        const double z = th * th;
        double p = -1.0 / 1307674368000.0;                  // -1/15!
        p = fma(p, z, 1.0 / 6227020800.0);                  //  1/13!
        p = fma(p, z, -1.0 / 39916800.0);                   // -1/11!
        p = fma(p, z, 1.0 / 362880.0);                      //  1/9!
        p = fma(p, z, -1.0 / 5040.0);                       // -1/7!
        p = fma(p, z, 1.0 / 120.0);                         //  1/5!
        p = fma(p, z, -1.0 / 6.0);                          // -1/3!
        *s = fma(th * z, p, th);
        double q = 1.0 / 20922789888000.0;                  //  1/16!
        q = fma(q, z, -1.0 / 87178291200.0);                // -1/14!
        q = fma(q, z, 1.0 / 479001600.0);                   //  1/12!
        q = fma(q, z, -1.0 / 3628800.0);                    // -1/10!
        q = fma(q, z, 1.0 / 40320.0);                       //  1/8!
        q = fma(q, z, -1.0 / 720.0);                        // -1/6!
        q = fma(q, z, 1.0 / 24.0);                          //  1/4!
        q = fma(q, z, -0.5);                                // -1/2!
        *c = fma(q, z, 1.0);
    } else {
        sincos(th, s, c);
    }
}

// One end of a branch seen from its own bus u towards bus v:
//   P = Gss Vu^2 + Vu Vv A,  Q = -Bss Vu^2 + Vu Vv C,  A = G cos th_u + B sin th_u,
//   C = G sin th_u - B cos th_u,  th_u = Va_u - Va_v.
struct End {
    double P, Q;
    double pa, pu, pv;   // dP / d(Va_u, Vm_u, Vm_v); dP/dVa_v = -pa
    double qa, qu, qv;   // dQ / d(Va_u, Vm_u, Vm_v)
};

template <bool DERIV>
__device__ __forceinline__ End end_terms(double Gss, double Bss, double A, double C, double Vu,
                                         double Vv) {
    End e;
    double GV = Gss * Vu, BV = Bss * Vu;
    double Ta = fma(Vv, A, GV);    // Gss Vu + Vv A
    double Tc = fma(Vv, C, -BV);   // -Bss Vu + Vv C
    e.P = Vu * Ta;
    e.Q = Vu * Tc;
    if (DERIV) {
        e.pu = Ta + GV;            // 2 Gss Vu + Vv A
        e.qu = Tc - BV;            // -2 Bss Vu + Vv C
        e.pv = Vu * A;
        e.qv = Vu * C;
        e.pa = -(Vv * e.qv);       // -Vu Vv C
        e.qa = Vv * e.pv;          //  Vu Vv A
    }
    return e;
}

// Distinct values of one end's Lagrangian Hessian block
//   lamP grad^2 P + lamQ grad^2 Q + mu grad^2 (P^2 + Q^2)   in (Va_u, Va_v, Vm_u, Vm_v):
//   (Va_u,Va_u) = -(Va_u,Va_v) = (Va_v,Va_v) = haa;  (Va_u,Vm_u) = -(Va_v,Vm_u) = hau;
//   (Va_u,Vm_v) = -(Va_v,Vm_v) = hav;  (Vm_u,Vm_u) = huu;  (Vm_u,Vm_v) = huv;  (Vm_v,Vm_v) = hvv.
struct EndHess {
    double haa, hau, hav, huu, huv, hvv;
};

__device__ __forceinline__ EndHess end_hess(const End &e, double Gss, double Bss, double A,
                                            double C, double K, double Vu, double Vv, double VV,
                                            double VV2, double lamP, double lamQ, double mu) {
    EndHess h;
    double mu2 = mu + mu;
    double wP = fma(mu2, e.P, lamP);              // multiplier of grad^2 P
    double wQ = fma(mu2, e.Q, lamQ);
    double W1 = fma(wP, A, wQ * C);
    double W2 = fma(wQ, A, -(wP * C));
    double E = fma(A, e.qu, -(C * e.pu));
    double F = fma(e.pu, A, e.qu * C);
    double tK = mu2 * K;                          // 2 mu (A^2 + C^2)
    h.haa = fma(tK, VV2, -(VV * W1));
    h.hau = fma(mu2 * VV, E, Vv * W2);
    h.hav = Vu * W2;
    double S = fma(e.pu, e.pu, e.qu * e.qu);
    double in = fma(wP, Gss, -(wQ * Bss));
    h.huu = fma(mu2, S, in + in);
    h.huv = fma(mu2 * Vu, F, W1);
    h.hvv = tK * (Vu * Vu);
    return h;
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
    double P2 = e.P + e.P, Q2 = e.Q + e.Q;
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

// One (state b, branch l) item.  scr is state b's slot-partial scratch ([NCOMP][nslot_pad]) and
// offs its parallel-branch scratch ([NOFF][nshared]).
template <int WANT>
__device__ __forceinline__ void branch_item(const DevNet &N, const EvalReq &R, int b, int l,
                                            double *scr, double *offs_base) {
    constexpr bool WG = WANT & W_G, WJ = WANT & W_J, WH = WANT & W_H;
    constexpr bool DERIV = WJ || WH;
    const int nb = N.nb, nl = N.nl;
    const size_t pad = (size_t)N.nslot_pad;
    const int sf = __ldg(N.br_slot + l), st = __ldg(N.br_slot + nl + l);
    const int fb = __ldg(N.f + l), tb = __ldg(N.t + l);
    const int sh = N.nshared ? __ldg(N.br_shared + l) : -1;
    double *Jb = WJ ? R.jval + (size_t)b * N.nnzJ : nullptr;
    double *Hb = WH ? R.hval + (size_t)b * N.nnzH : nullptr;
    double *offs = sh >= 0 ? offs_base + sh : nullptr;
    auto put_off = [&](int c, double v, double *base) {
        if (sh >= 0) offs[(size_t)c * N.nshared] = v;
        else base[__ldg(N.br_off + (size_t)c * nl + l)] = v;
    };
    double *Jf = WJ ? Jb + N.nnzJg + 4 * (size_t)l : nullptr;
    double *Jt = WJ ? Jb + N.nnzJg + 4 * (size_t)nl + 4 * (size_t)l : nullptr;
    double *ghb = R.gh ? R.gh + (size_t)b * N.m : nullptr;

    const bool on = R.mask == nullptr || R.mask[(size_t)b * nl + l] != 0;
    if (!on) {   // out of service: every value of this branch is zero
        scr[SC_P * pad + sf] = 0.0; scr[SC_Q * pad + sf] = 0.0;
        scr[SC_P * pad + st] = 0.0; scr[SC_Q * pad + st] = 0.0;
        if (WG && ghb) { ghb[2 * nb + l] = 0.0; ghb[2 * nb + nl + l] = 0.0; }
        if (WJ) {
            for (int c = SC_PA; c <= SC_QU; c++) { scr[c * pad + sf] = 0.0; scr[c * pad + st] = 0.0; }
            for (int c = OJ_PF_VAT; c <= OJ_QT_VMF; c++) put_off(c, 0.0, Jb);
            for (int k = 0; k < 4; k++) { Jf[k] = 0.0; Jt[k] = 0.0; }
        }
        if (WH) {
            for (int c = SC_HAA; c <= SC_HUU; c++) { scr[c * pad + sf] = 0.0; scr[c * pad + st] = 0.0; }
            for (int c = OH_AA; c <= OH_MT_AF; c++) put_off(c, 0.0, Hb);
        }
        return;
    }

    const double *xb = R.x + (size_t)b * N.n;
    const double Vaf = __ldg(xb + fb), Vat = __ldg(xb + tb);
    const double Vf = __ldg(xb + nb + fb), Vt = __ldg(xb + nb + tb);
    const double G = __ldg(N.Gft + l), Bm = __ldg(N.Bft + l);
    const double Gff = __ldg(N.Gff + l), Bff = __ldg(N.Bff + l);
    const double Gtt = __ldg(N.Gtt + l), Btt = __ldg(N.Btt + l);

    double s, c;
    branch_sincos(Vaf - Vat, &s, &c);
    const double Gc = G * c, Gs = G * s, Bc = Bm * c, Bs = Bm * s;
    const double Af = Gc + Bs, Cf = Gs - Bc;          // from end, th = Va_f - Va_t
    const double At = Gc - Bs, Ct = -(Gs + Bc);       // to end,   th = Va_t - Va_f

    const End ef = end_terms<DERIV>(Gff, Bff, Af, Cf, Vf, Vt);
    const End et = end_terms<DERIV>(Gtt, Btt, At, Ct, Vt, Vf);

    scr[SC_P * pad + sf] = ef.P; scr[SC_Q * pad + sf] = ef.Q;
    scr[SC_P * pad + st] = et.P; scr[SC_Q * pad + st] = et.Q;
    if (WG && ghb) {
        ghb[2 * nb + l] = fma(ef.P, ef.P, ef.Q * ef.Q);
        ghb[2 * nb + nl + l] = fma(et.P, et.P, et.Q * et.Q);
    }
    if (WJ) {
        scr[SC_PA * pad + sf] = ef.pa; scr[SC_PU * pad + sf] = ef.pu;
        scr[SC_QA * pad + sf] = ef.qa; scr[SC_QU * pad + sf] = ef.qu;
        scr[SC_PA * pad + st] = et.pa; scr[SC_PU * pad + st] = et.pu;
        scr[SC_QA * pad + st] = et.qa; scr[SC_QU * pad + st] = et.qu;
        put_off(OJ_PF_VAT, dneg(ef.pa), Jb); put_off(OJ_PF_VMT, ef.pv, Jb);
        put_off(OJ_QF_VAT, dneg(ef.qa), Jb); put_off(OJ_QF_VMT, ef.qv, Jb);
        put_off(OJ_PT_VAF, dneg(et.pa), Jb); put_off(OJ_PT_VMF, et.pv, Jb);
        put_off(OJ_QT_VAF, dneg(et.qa), Jb); put_off(OJ_QT_VMF, et.qv, Jb);
        store_hrow(Jf, ef, fb < tb);
        store_hrow(Jt, et, tb < fb);
    }
    if (WH) {
        const double *lb = R.lam + (size_t)b * N.m;
        const double lPf = __ldg(lb + fb), lPt = __ldg(lb + tb);
        const double lQf = __ldg(lb + nb + fb), lQt = __ldg(lb + nb + tb);
        const double muf = __ldg(lb + 2 * nb + l), mut = __ldg(lb + 2 * nb + nl + l);
        const double K = fma(G, G, Bm * Bm);          // A^2 + C^2 at both ends
        const double VV = Vf * Vt, VV2 = VV * VV;
        const EndHess hf = end_hess(ef, Gff, Bff, Af, Cf, K, Vf, Vt, VV, VV2, lPf, lQf, muf);
        const EndHess ht = end_hess(et, Gtt, Btt, At, Ct, K, Vt, Vf, VV, VV2, lPt, lQt, mut);
        const double haa = hf.haa + ht.haa;
        const double xf = hf.hau - ht.hav;            // (Vm_f, Va_f)
        const double xt = ht.hau - hf.hav;            // (Vm_t, Va_t)
        scr[SC_HAA * pad + sf] = haa; scr[SC_HAA * pad + st] = haa;
        scr[SC_HUA * pad + sf] = xf;  scr[SC_HUA * pad + st] = xt;
        scr[SC_HUU * pad + sf] = hf.huu + ht.hvv;
        scr[SC_HUU * pad + st] = ht.huu + hf.hvv;
        put_off(OH_AA, dneg(haa), Hb);
        put_off(OH_MM, hf.huv + ht.huv, Hb);
        put_off(OH_MF_AT, dneg(xf), Hb);
        put_off(OH_MT_AF, dneg(xt), Hb);
    }
}

// Gradient entry of generator k's active power: w (2 c2 base^2 Pg + c1 base).
__device__ __forceinline__ double grad_pg(const DevNet &N, const EvalReq &R, int b, int k) {
    const double w = R.obj_weight ? R.obj_weight[b] : 1.0;
    const double base = N.baseMVA;
    const double Pg = __ldg(R.x + (size_t)b * N.n + 2 * N.nb + k);
    return w * fma(2.0 * __ldg(N.c2 + k) * base * base, Pg, __ldg(N.c1 + k) * base);
}

// One (state b, bus i) item: sums the bus's branch-end partials in slot order, adds shunt, load
// and generator terms, and writes the bus's g rows, its diagonal J and H values and its
// generators' constant J entries and cost Hessian.  The partials are read through L2 (ld.cg):
// in the persistent schedule other CTAs wrote them during the same launch.
template <int WANT>
__device__ __forceinline__ void bus_item(const DevNet &N, const EvalReq &R, int b, int i,
                                         const double *scr) {
    constexpr bool WG = WANT & W_G, WJ = WANT & W_J, WH = WANT & W_H;
    const int nb = N.nb;
    const size_t pad = (size_t)N.nslot_pad;
    const int s0 = __ldg(N.slot_ptr + i), s1 = __ldg(N.slot_ptr + i + 1);
    const int g0 = __ldg(N.gen_ptr + i), g1 = __ldg(N.gen_ptr + i + 1);
    const double *xb = R.x + (size_t)b * N.n;
    const double Vm = __ldg(xb + nb + i);
    const double Gs = __ldg(N.Gs + i), Bs = __ldg(N.Bs + i);

    if (WG && R.gh) {
        double sP = 0.0, sQ = 0.0;
        for (int s = s0; s < s1; s++) {
            sP += __ldcg(scr + SC_P * pad + s);
            sQ += __ldcg(scr + SC_Q * pad + s);
        }
        const double sc = R.pd_scale ? __ldg(R.pd_scale + (size_t)b * nb + i) : 1.0;
        const double VV = Vm * Vm;
        sP += fma(Gs, VV, __ldg(N.Pd + i) * sc);
        sQ += fma(-Bs, VV, __ldg(N.Qd + i) * sc);
        for (int s = g0; s < g1; s++) {
            const int k = __ldg(N.gen_ord + s);
            sP -= __ldg(xb + 2 * nb + k);
            sQ -= __ldg(xb + 2 * nb + N.ng + k);
        }
        double *ghb = R.gh + (size_t)b * N.m;
        ghb[i] = sP;
        ghb[nb + i] = sQ;
    }
    if (WJ) {
        double pa = 0.0, pu = 0.0, qa = 0.0, qu = 0.0;
        for (int s = s0; s < s1; s++) {
            pa += __ldcg(scr + SC_PA * pad + s); pu += __ldcg(scr + SC_PU * pad + s);
            qa += __ldcg(scr + SC_QA * pad + s); qu += __ldcg(scr + SC_QU * pad + s);
        }
        const double tV = Vm + Vm;
        pu = fma(Gs, tV, pu);
        qu = fma(-Bs, tV, qu);
        double *Jb = R.jval + (size_t)b * N.nnzJ;
        const int jP = __ldg(N.bus_jP + i), jQ = __ldg(N.bus_jQ + i), k = __ldg(N.bus_k + i);
        Jb[jP] = pa; Jb[jP + k] = pu;
        Jb[jQ] = qa; Jb[jQ + k] = qu;
        for (int s = g0; s < g1; s++) {
            const int g = __ldg(N.gen_ord + s);
            Jb[__ldg(N.gen_jP + g)] = -1.0;
            Jb[__ldg(N.gen_jQ + g)] = -1.0;
        }
    }
    if (WH) {
        double aa = 0.0, ua = 0.0, uu = 0.0;
        for (int s = s0; s < s1; s++) {
            aa += __ldcg(scr + SC_HAA * pad + s);
            ua += __ldcg(scr + SC_HUA * pad + s);
            uu += __ldcg(scr + SC_HUU * pad + s);
        }
        const double *lb = R.lam + (size_t)b * N.m;
        const double lP = __ldg(lb + i), lQ = __ldg(lb + nb + i);
        uu += fma(lP, Gs + Gs, -(lQ * (Bs + Bs)));
        double *Hb = R.hval + (size_t)b * N.nnzH;
        Hb[__ldg(N.bus_h + i)] = aa;
        Hb[__ldg(N.bus_h + nb + i)] = ua;
        Hb[__ldg(N.bus_h + 2 * nb + i)] = uu;
        if (g1 > g0) {
            const double sw = R.sigma * (R.obj_weight ? R.obj_weight[b] : 1.0);
            const double base2 = N.baseMVA * N.baseMVA;
            for (int s = g0; s < g1; s++) {
                const int g = __ldg(N.gen_ord + s);
                Hb[__ldg(N.gen_h + g)] = sw * (2.0 * __ldg(N.c2 + g) * base2);
            }
        }
    }
}

// Gradient entries owned by bus i: Va_i and Vm_i (zero) and, for each generator at i, Pg and Qg.
__device__ __forceinline__ void grad_bus(const DevNet &N, const EvalReq &R, int b, int i) {
    double *gb = R.grad + (size_t)b * N.n;
    gb[i] = 0.0;
    gb[N.nb + i] = 0.0;
    const int g0 = __ldg(N.gen_ptr + i), g1 = __ldg(N.gen_ptr + i + 1);
    for (int s = g0; s < g1; s++) {
        const int k = __ldg(N.gen_ord + s);
        gb[2 * N.nb + k] = grad_pg(N, R, b, k);
        gb[2 * N.nb + N.ng + k] = 0.0;
    }
}

// Parallel-branch fixup entry e of state b: sums the group's values in ascending branch order.
__device__ __forceinline__ void fixup_entry(const DevNet &N, const EvalReq &R, int b, int e,
                                            const double *offs) {
    const bool isH = N.fix_isH[e] != 0;
    if ((isH && !R.hval) || (!isH && !R.jval)) return;
    double v = 0.0;
    for (int p = N.fix_ptr[e]; p < N.fix_ptr[e + 1]; p++) v += __ldcg(offs + N.fix_src[p]);
    if (isH) R.hval[(size_t)b * N.nnzH + N.fix_dst[e]] = v;
    else R.jval[(size_t)b * N.nnzJ + N.fix_dst[e]] = v;
}

// Objective of state b, f = w sum_k (c2 MW^2 + c1 MW + c0), MW = base Pg, by the whole block.
// Virtual lane v < 256 sums generators v, v+256, ... in order; the 256 partials are combined by
// a fixed pairwise tree.  The result is the same for every block size.  part: 256 doubles of
// shared memory.
constexpr int OBJ_LANES = 256;
__device__ __forceinline__ void obj_block(const DevNet &N, const EvalReq &R, int b, double *part) {
    const double *Pg = R.x + (size_t)b * N.n + 2 * N.nb;
    for (int v = threadIdx.x; v < OBJ_LANES; v += blockDim.x) {
        double acc = 0.0;
        for (int k = v; k < N.ng; k += OBJ_LANES) {
            const double MW = N.baseMVA * __ldg(Pg + k);
            acc += fma(fma(__ldg(N.c2 + k), MW, __ldg(N.c1 + k)), MW, __ldg(N.c0 + k));
        }
        part[v] = acc;
    }
    __syncthreads();
    for (int w = OBJ_LANES / 2; w > 0; w >>= 1) {
        for (int v = threadIdx.x; v < w; v += blockDim.x) part[v] += part[v + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) R.f[b] = (R.obj_weight ? R.obj_weight[b] : 1.0) * part[0];
    __syncthreads();
}


// Records an event on the launching stream before a kernel when profiling.
static inline void mark(ProfileHook *hk, cudaStream_t st, const char *name) {
    if (!hk || hk->n >= ProfileHook::MAX - 1) return;
    cudaEventRecord(hk->ev[hk->n], st);
    hk->name[hk->n] = name;
    hk->n++;
}

}  // namespace exago
