// The power-balance-cartesian formulation of the AC-OPF model, which ExaGO offers beside the polar
// one (arXiv 2203.10587, Sec. III): the bus voltage is V_i = e_i + j f_i, the variables are
// x = [e | f | Pg | Qg], and the voltage-magnitude limits become rows e_i^2 + f_i^2 after the
// flow rows, so that g | h = [P balance | Q balance | |S_from|^2 | |S_to|^2 | e^2 + f^2] and the
// multipliers are [lamP | lamQ | muF | muT | muV].
//
// For one end of a branch, from its bus u towards v, with a = e_u e_v + f_u f_v,
// b = f_u e_v - e_u f_v and s = e_u^2 + f_u^2:
//     P = Gss s + G a + B b,     Q = -Bss s + G b - B a.
// Both are quadratic forms, so every derivative is a product of admittances and voltages (no sine
// or cosine), the second derivatives of P and Q are constants, and dQ/de_v = dP/df_v,
// dQ/df_v = -dP/de_v.
//
// The J rows of g and h and the Hessian have the polar model's sparsity pattern with e in place of
// Va and f in place of Vm, so the kernels reuse the net's plan (row starts, slot order, positions);
// the nb voltage rows follow the polar rows in the Jacobian (entries 2 e_i, 2 f_i).  Schedule: per
// chunk of states, a branch kernel writes each branch end's 14-value record at its slot and the
// branch's h values and h rows; a bus kernel walks each bus's slots in the plan's fixed order,
// writes the neighbour entries of its J and H rows and finishes the diagonal, balance, voltage
// and generator terms.  The branch kernel of the next chunk runs on the caller's stream while the
// bus kernel of the previous one runs on the net's side stream (ordered by events only), with a
// ring of three chunks of records sized to stay in L2; each kernel's grid is its resident CTA
// count, looping over (state, block) work items.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "eval_items.cuh"
#include "persist_kernel.cuh"

namespace exago {
namespace {

// One branch-end record (end at bus u towards bus v).
enum CartComp {
    CR_P = 0, CR_Q = 1,                        // injections
    CR_PE = 2, CR_PF = 3, CR_QE = 4, CR_QF = 5,   // dP/de_u, dP/df_u, dQ/de_u, dQ/df_u
    CR_PEV = 6, CR_PFV = 7,                    // dP/de_v, dP/df_v (dQ/de_v = dP/df_v, dQ/df_v = -dP/de_v)
    CR_HEE = 8, CR_HFE = 9, CR_HFF = 10,       // branch Hessian (e_u,e_u), (f_u,e_u), (f_u,f_u)
    CR_HEEV = 11, CR_HFEV = 12, CR_HFFV = 13,  // (e_u,e_v), (f_u,e_v), (f_u,f_v)
    CNC = 14
};

// Records of one chunk of states; a ring of kRing chunks (72 MiB) stays in L2 between the branch
// kernel that writes a chunk and the bus kernel that reads it.
constexpr size_t kChunkRecordBytes = (size_t)24 << 20;
constexpr int kRing = 3;
// Branch values of one chunk of states in the adjoint products (one stream, no ring).
constexpr size_t kAdjChunkBytes = (size_t)48 << 20;

struct CartReq {
    int B, b0;                  // states of this launch: b0 .. b0 + nB (the kernels' argument)
    int mc;                     // rows of g | h: m + nb
    int64_t nnzJc;              // Jacobian entries per state: nnzJ + 2 nb
    const double *x, *lam;
    const uint8_t *mask, *gen_mask;
    const double *pd_scale, *obj_weight;
    double sigma;
    double *f, *grad, *gh, *jval, *hval;
    double *scratch;            // [chunk][nslot][CNC]
    int stage_cap;              // persistent schedule: shared-memory doubles of a bus tile's rows
};

// Output stores: written once and never read by the kernels, so they are marked evict-first
// (st.global.cs) and leave L2 to the branch-end records, which are read back.
__device__ __forceinline__ void out(double *p, double v) { __stcs(p, v); }

__device__ __forceinline__ void put2c(double *rec, int c, double a, double b) {
    *reinterpret_cast<double2 *>(rec + c) = make_double2(a, b);
}

// Flows and first derivatives of one branch at voltages (ef + j ff, et + j ft).  For the end at u
// towards v, p = dP/d(e_u, f_u, e_v, f_v) and q1, q2 = dQ/d(e_u, f_u); dQ/de_v = p4, dQ/df_v = -p3.
struct CartBranch {
    double Pf, Qf, Pt, Qt;
    double p1f, p2f, q1f, q2f, p3f, p4f;   // from end (u = f, v = t)
    double p1t, p2t, q1t, q2t, p3t, p4t;   // to end (u = t, v = f)
};

// The admittances of one branch (network tables).  G, Bm are the from end's mutual admittance;
// Gt, Bt the to end's, read only by the phase-shifter variants (PS; equal to G, Bm otherwise).
struct CartY {
    double G, Bm, Gff, Bff, Gtt, Btt, Gff2, Bff2, Gtt2, Btt2, Gt, Bt;
};

template <bool PS>
__device__ __forceinline__ CartY cart_y(const DevNet &N, int l) {
    CartY y;
    y.G = __ldg(N.Gft + l); y.Bm = __ldg(N.Bft + l);
    if (PS) { y.Gt = __ldg(N.Gtf + l); y.Bt = __ldg(N.Btf + l); }
    else { y.Gt = y.G; y.Bt = y.Bm; }
    y.Gff = __ldg(N.Gff + l); y.Bff = __ldg(N.Bff + l);
    y.Gtt = __ldg(N.Gtt + l); y.Btt = __ldg(N.Btt + l);
    y.Gff2 = __ldg(N.Gff2 + l); y.Bff2 = __ldg(N.Bff2 + l);
    y.Gtt2 = __ldg(N.Gtt2 + l); y.Btt2 = __ldg(N.Btt2 + l);
    return y;
}

// With PS (phase-shifting transformers) the to end's terms take its own mutual admittance
// (Gt, Bt); without, Gt = G and Bt = Bm and the products of Bm with the four voltage components
// serve both ends.  The mutual parts of the injections are linear in the far end's voltage, so
// with u = d(G a + B b)/d(e_f, f_f) and w = d(G a - B b)/d(e_t, f_t) (a = e_f e_t + f_f f_t,
// b = f_f e_t - e_f f_t):  G a + B b = e_f u1 + f_f u2,  G b - B a = f_f u1 - e_f u2,  and at
// the to end  G a - B b = e_t w1 + f_t w2,  -(G b + B a) = f_t w1 - e_t w2.
template <bool PS>
__device__ __forceinline__ CartBranch cart_terms(const CartY &y, double ef, double ff, double et,
                                                 double ft) {
    const double G = y.G, Bm = y.Bm, Gff = y.Gff, Bff = y.Bff, Gtt = y.Gtt, Btt = y.Btt;
    const double Gff2 = y.Gff2, Bff2 = y.Bff2, Gtt2 = y.Gtt2, Btt2 = y.Btt2;
    CartBranch c;
    const double sf = fma(ef, ef, ff * ff), st = fma(et, et, ft * ft);
    const double Bef = Bm * ef, Bff_ = Bm * ff, Bet = Bm * et, Bft_ = Bm * ft;
    const double u1 = fma(G, et, -Bft_), u2 = fma(G, ft, Bet);
    c.p3f = fma(G, ef, Bff_); c.p4f = fma(G, ff, -Bef);          // dP_f/d(e_t, f_t)
    double w1, w2;
    if (PS) {
        const double Gt = y.Gt, Bt = y.Bt;
        const double Btef = Bt * ef, Btff = Bt * ff, Btet = Bt * et, Btft = Bt * ft;
        w1 = fma(Gt, ef, -Btff); w2 = fma(Gt, ff, Btef);
        c.p3t = fma(Gt, et, Btft); c.p4t = fma(Gt, ft, -Btet);   // dP_t/d(e_f, f_f)
    } else {
        w1 = fma(G, ef, -Bff_); w2 = fma(G, ff, Bef);
        c.p3t = fma(G, et, Bft_); c.p4t = fma(G, ft, -Bet);
    }
    c.Pf = fma(Gff, sf, fma(ef, u1, ff * u2));
    c.Qf = fma(-Bff, sf, fma(ff, u1, -(ef * u2)));
    c.Pt = fma(Gtt, st, fma(et, w1, ft * w2));
    c.Qt = fma(-Btt, st, fma(ft, w1, -(et * w2)));
    c.p1f = fma(Gff2, ef, u1); c.p2f = fma(Gff2, ff, u2);
    c.q1f = fma(-Bff2, ef, -u2); c.q2f = fma(-Bff2, ff, u1);
    c.p1t = fma(Gtt2, et, w1); c.p2t = fma(Gtt2, ft, w2);
    c.q1t = fma(-Btt2, et, -w2); c.q2t = fma(-Btt2, ft, w1);
    return c;
}

// The branch's Lagrangian-Hessian block over (e_f, f_f, e_t, f_t), 10 distinct values.  End
// weights wP = lamP + 2 mu P, wQ = lamQ + 2 mu Q; the linear part of each end's block is
// wP grad^2 P + wQ grad^2 Q: d = 2 (wP Gss - wQ Bss) on (e_u,e_u) and (f_u,f_u),
// c1 = wP G - wQ B on (e_u,e_v) and (f_u,f_v), c2 = wP B + wQ G on (f_u,e_v) and -c2 on (e_u,f_v).
// The rest is O = 2 mu (grad P grad P' + grad Q grad Q') of each end; with q3 = p4, q4 = -p3 its
// (e_v,e_v) and (f_v,f_v) entries are both 2 mu (p3^2 + p4^2) and its (f_v,e_v) entry vanishes.
// The gradients are scaled by 2 mu once, and each entry is one chain of fused multiply-adds.
struct CartHess {
    double eef, fef, fff;            // (e_f,e_f), (f_f,e_f), (f_f,f_f)
    double eet, fet, fft;            // (e_t,e_t), (f_t,e_t), (f_t,f_t)
    double eeft, ffft, ef_ft, ff_et; // (e_f,e_t), (f_f,f_t), (e_f,f_t), (f_f,e_t)
};

template <bool PS>
__device__ __forceinline__ CartHess cart_hess(const CartY &y, const CartBranch &c, double lPf,
                                              double lQf, double lPt, double lQt, double muf,
                                              double mut) {
    const double G = y.G, Bm = y.Bm, Gff2 = y.Gff2, Bff2 = y.Bff2, Gtt2 = y.Gtt2, Btt2 = y.Btt2;
    const double muf2 = twice(muf), mut2 = twice(mut);
    const double wPf = fma(muf2, c.Pf, lPf), wQf = fma(muf2, c.Qf, lQf);
    const double wPt = fma(mut2, c.Pt, lPt), wQt = fma(mut2, c.Qt, lQt);
    const double df = fma(wPf, Gff2, -(wQf * Bff2)), dt = fma(wPt, Gtt2, -(wQt * Btt2));
    double c1, dc;
    if (PS) {   // each end with its own mutual admittance
        c1 = fma(wPf, G, fma(wPt, y.Gt, -fma(wQf, Bm, wQt * y.Bt)));        // c1_f + c1_t
        dc = fma(wPt, y.Bt, fma(wQt, y.Gt, -fma(wPf, Bm, wQf * G)));        // c2_t - c2_f
    } else {
        c1 = fma(wPf + wPt, G, -((wQf + wQt) * Bm));                        // c1_f + c1_t
        dc = fma(wPt - wPf, Bm, (wQt - wQf) * G);                           // c2_t - c2_f
    }
    // 2 mu times each end's gradient
    const double a1 = muf2 * c.p1f, a2 = muf2 * c.p2f, a3 = muf2 * c.p3f, a4 = muf2 * c.p4f;
    const double b1 = muf2 * c.q1f, b2 = muf2 * c.q2f;
    const double s1 = mut2 * c.p1t, s2 = mut2 * c.p2t, s3 = mut2 * c.p3t, s4 = mut2 * c.p4t;
    const double r1 = mut2 * c.q1t, r2 = mut2 * c.q2t;
    CartHess h;
    const double dfo = df + fma(s3, c.p3t, s4 * c.p4t);   // d_f + (e_t,e_t) block of O_t
    const double dto = dt + fma(a3, c.p3f, a4 * c.p4f);
    h.eef = fma(a1, c.p1f, fma(b1, c.q1f, dfo));
    h.fef = fma(a2, c.p1f, b2 * c.q1f);
    h.fff = fma(a2, c.p2f, fma(b2, c.q2f, dfo));
    h.eet = fma(s1, c.p1t, fma(r1, c.q1t, dto));
    h.fet = fma(s2, c.p1t, r2 * c.q1t);
    h.fft = fma(s2, c.p2t, fma(r2, c.q2t, dto));
    h.eeft = fma(a1, c.p3f, fma(b1, c.p4f, fma(s1, c.p3t, fma(r1, c.p4t, c1))));
    h.ffft = fma(a2, c.p4f, fma(-b2, c.p3f, fma(s2, c.p4t, fma(-r2, c.p3t, c1))));
    h.ef_ft = fma(a1, c.p4f, fma(-b1, c.p3f, fma(s2, c.p3t, fma(r2, c.p4t, dc))));
    h.ff_et = fma(a2, c.p3f, fma(b2, c.p4f, fma(s1, c.p4t, fma(-r1, c.p3t, -dc))));
    return h;
}

// One (state b, branch l) item: scr is state b's records ([nslot][CNC]).
template <bool PS>
__device__ __forceinline__ void cart_branch_item_at(const DevNet &N, const CartReq &R, int b,
                                                    double *scr, int l) {
    const int nb = N.nb, nl = N.nl;
    double *rf = scr + (size_t)__ldg(N.br_slot + l) * CNC;
    double *rt = scr + (size_t)__ldg(N.br_slot + nl + l) * CNC;
    const int fb = __ldg(N.f + l), tb = __ldg(N.t + l);
    double *ghb = R.gh ? R.gh + (size_t)b * R.mc : nullptr;
    double *Jf = R.jval ? R.jval + (size_t)b * R.nnzJc + N.nnzJg + 4 * (size_t)l : nullptr;
    double *Jt = Jf ? Jf + 4 * (size_t)nl : nullptr;
    const bool on = R.mask == nullptr || R.mask[(size_t)b * nl + l] != 0;
    if (!on) {
#pragma unroll
        for (int c = 0; c < CNC; c += 2) { put2c(rf, c, 0.0, 0.0); put2c(rt, c, 0.0, 0.0); }
        if (ghb) { out(ghb + 2 * nb + l, 0.0); out(ghb + 2 * nb + nl + l, 0.0); }
        if (Jf)
            for (int k = 0; k < 4; k++) { out(Jf + k, 0.0); out(Jt + k, 0.0); }
        return;
    }
    const double *xb = R.x + (size_t)b * N.n;
    const CartY y = cart_y<PS>(N, l);
    const CartBranch c = cart_terms<PS>(y, __ldg(xb + fb), __ldg(xb + nb + fb), __ldg(xb + tb),
                                        __ldg(xb + nb + tb));
    if (ghb) {
        out(ghb + 2 * nb + l, fma(c.Pf, c.Pf, c.Qf * c.Qf));
        out(ghb + 2 * nb + nl + l, fma(c.Pt, c.Pt, c.Qt * c.Qt));
    }
    if (Jf) {
        // grad |S|^2 = 2 P grad P + 2 Q grad Q, columns (e_lo, e_hi, f_lo, f_hi)
        const double Pf2 = twice(c.Pf), Qf2 = twice(c.Qf), Pt2 = twice(c.Pt), Qt2 = twice(c.Qt);
        const double hff_e = fma(Pf2, c.p1f, Qf2 * c.q1f), hff_f = fma(Pf2, c.p2f, Qf2 * c.q2f);
        const double hft_e = fma(Pf2, c.p3f, Qf2 * c.p4f), hft_f = fma(Pf2, c.p4f, -(Qf2 * c.p3f));
        const double htt_e = fma(Pt2, c.p1t, Qt2 * c.q1t), htt_f = fma(Pt2, c.p2t, Qt2 * c.q2t);
        const double htf_e = fma(Pt2, c.p3t, Qt2 * c.p4t), htf_f = fma(Pt2, c.p4t, -(Qt2 * c.p3t));
        if (fb < tb) {
            out(Jf, hff_e); out(Jf + 1, hft_e); out(Jf + 2, hff_f); out(Jf + 3, hft_f);
            out(Jt, htf_e); out(Jt + 1, htt_e); out(Jt + 2, htf_f); out(Jt + 3, htt_f);
        } else {
            out(Jf, hft_e); out(Jf + 1, hff_e); out(Jf + 2, hft_f); out(Jf + 3, hff_f);
            out(Jt, htt_e); out(Jt + 1, htf_e); out(Jt + 2, htt_f); out(Jt + 3, htf_f);
        }
    }
    put2c(rf, CR_P, c.Pf, c.Qf);
    put2c(rf, CR_PE, c.p1f, c.p2f);
    put2c(rf, CR_QE, c.q1f, c.q2f);
    put2c(rf, CR_PEV, c.p3f, c.p4f);
    put2c(rt, CR_P, c.Pt, c.Qt);
    put2c(rt, CR_PE, c.p1t, c.p2t);
    put2c(rt, CR_QE, c.q1t, c.q2t);
    put2c(rt, CR_PEV, c.p3t, c.p4t);
    if (R.hval) {
        const double *lb = R.lam + (size_t)b * R.mc;
        const CartHess h = cart_hess<PS>(y, c, __ldg(lb + fb), __ldg(lb + nb + fb), __ldg(lb + tb),
                                         __ldg(lb + nb + tb), __ldg(lb + 2 * nb + l),
                                         __ldg(lb + 2 * nb + nl + l));
        put2c(rf, CR_HEE, h.eef, h.fef);
        put2c(rf, CR_HFF, h.fff, h.eeft);
        put2c(rf, CR_HFEV, h.ff_et, h.ffft);
        put2c(rt, CR_HEE, h.eet, h.fet);
        put2c(rt, CR_HFF, h.fft, h.eeft);
        put2c(rt, CR_HFEV, h.ef_ft, h.ffft);
    }
}

// Work items (state of the chunk, block of 128 branches or buses), state-major, taken by a grid
// of the resident CTA count so that no launch ends in a nearly empty wave.
// PS: the net has phase-shifting transformers (N.Gtf non-null).
template <bool PS>
__global__ void __launch_bounds__(128) k_cart_branch(const DevNet N, const CartReq R, int nB) {
    const int per = (N.nl + 127) / 128;
    for (int it = blockIdx.x; it < nB * per; it += gridDim.x) {
        const int bl = it / per;
        const int l = (it - bl * per) * 128 + threadIdx.x;
        if (l < N.nl)
            cart_branch_item_at<PS>(N, R, R.b0 + bl, R.scratch + (size_t)bl * N.nslot * CNC, l);
    }
}

// The values a bus reads from one record.
struct CRec {
    double P, Q, pe, pf, qe, qf, pev, pfv, hee, hfe, hff, heev, hfev, hffv;
};

__device__ __forceinline__ CRec load_crec(const double *r, bool wantH) {
    CRec o;
    double2 v = ld2(r + CR_P);
    o.P = v.x; o.Q = v.y;
    v = ld2(r + CR_PE); o.pe = v.x; o.pf = v.y;
    v = ld2(r + CR_QE); o.qe = v.x; o.qf = v.y;
    v = ld2(r + CR_PEV); o.pev = v.x; o.pfv = v.y;
    if (wantH) {
        v = ld2(r + CR_HEE); o.hee = v.x; o.hfe = v.y;
        v = ld2(r + CR_HFF); o.hff = v.x; o.heev = v.y;
        v = ld2(r + CR_HFEV); o.hfev = v.x; o.hffv = v.y;
    } else {
        o.hee = o.hfe = o.hff = o.heev = o.hfev = o.hffv = 0.0;
    }
    return o;
}

// Bus i's four rows (J rows P_i and Q_i, H rows e_i and f_i) in state b's outputs, or null
// where that output is not wanted.
__device__ __forceinline__ BusRows cart_rows(const DevNet &N, const CartReq &R, int b, int i) {
    BusRows W{};
    if (R.jval) {
        double *Jb = R.jval + (size_t)b * R.nnzJc;
        W.JP = Jb + __ldg(N.bus_jP + i);
        W.JQ = Jb + __ldg(N.bus_jQ + i);
    }
    if (R.hval) {
        double *Hb = R.hval + (size_t)b * N.nnzH;
        W.HA = Hb + __ldg(N.bus_hA + i);
        W.HM = Hb + __ldg(N.bus_hM + i);
    }
    return W;
}

// One (state b, bus i) item: scr is state b's records ([nslot][CNC]); W the bus's rows (in
// global memory or in a tile's shared-memory copy).
__device__ __forceinline__ void cart_bus_item_at(const DevNet &N, const CartReq &R, int b,
                                                 const double *scr, int i, const BusRows &W) {
    const int nb = N.nb, ng = N.ng;
    const bool wantH = R.hval != nullptr;
    const int s0 = __ldg(N.slot_ptr + i), s1 = __ldg(N.slot_ptr + i + 1);
    const int k = __ldg(N.bus_k + i), nlow = __ldg(N.bus_nlow + i);
    double *Jb = R.jval ? R.jval + (size_t)b * R.nnzJc : nullptr;
    double *Hb = wantH ? R.hval + (size_t)b * N.nnzH : nullptr;
    double *JP = W.JP, *JQ = W.JQ, *HA = W.HA, *HM = W.HM;

    // diagonal sums over the bus's ends, and one neighbour group (parallel branches) at a time
    double P = 0.0, Q = 0.0, pe = 0.0, pf = 0.0, qe = 0.0, qf = 0.0, hee = 0.0, hfe = 0.0, hff = 0.0;
    int pos = 0;
    int s = s0;
    while (s < s1) {
        const int j = __ldg(N.slot_nbr + s);
        CRec o = load_crec(scr + (size_t)s * CNC, wantH);
        P += o.P; Q += o.Q; pe += o.pe; pf += o.pf; qe += o.qe; qf += o.qf;
        hee += o.hee; hfe += o.hfe; hff += o.hff;
        for (s++; s < s1 && __ldg(N.slot_nbr + s) == j; s++) {
            const CRec p = load_crec(scr + (size_t)s * CNC, wantH);
            P += p.P; Q += p.Q; pe += p.pe; pf += p.pf; qe += p.qe; qf += p.qf;
            hee += p.hee; hfe += p.hfe; hff += p.hff;
            o.pev += p.pev; o.pfv += p.pfv; o.heev += p.heev; o.hfev += p.hfev; o.hffv += p.hffv;
        }
        if (pos == nlow) pos++;   // the diagonal column sits between lower and upper neighbours
        if (JP) {
            JP[pos] = o.pev; JP[k + pos] = o.pfv;              // dP/de_j, dP/df_j
            JQ[pos] = o.pfv; JQ[k + pos] = dneg(o.pev);        // dQ/de_j, dQ/df_j
        }
        if (HM) {
            HM[pos] = o.hfev;                                  // (f_i, e_j)
            if (j < i) {
                HA[pos] = o.heev;                              // (e_i, e_j)
                HM[k + pos] = o.hffv;                          // (f_i, f_j)
            }
        }
        pos++;
    }

    const double *xb = R.x + (size_t)b * N.n;
    const double ei = __ldg(xb + i), fi = __ldg(xb + nb + i);
    const double Gs = __ldg(N.Gs + i), Bs = __ldg(N.Bs + i);
    const double V2 = fma(ei, ei, fi * fi);
    const int g0 = __ldg(N.gen_ptr + i), g1 = __ldg(N.gen_ptr + i + 1);
    // generators out of service inject nothing and have zero entries
    const uint8_t *gm = R.gen_mask && g1 > g0 ? R.gen_mask + (size_t)b * ng : nullptr;
    if (R.gh) {
        double Pd = __ldg(N.Pd + i), Qd = __ldg(N.Qd + i);
        if (R.pd_scale) {
            const double sc = __ldg(R.pd_scale + (size_t)b * nb + i);
            Pd *= sc;
            Qd *= sc;
        }
        double gP = fma(Gs, V2, P) + Pd;
        double gQ = fma(-Bs, V2, Q) + Qd;
        for (int q = g0; q < g1; q++) {
            const int g = __ldg(N.gen_ord + q);
            if (!gen_on(gm, g)) continue;
            gP -= __ldg(xb + 2 * nb + g);
            gQ -= __ldg(xb + 2 * nb + ng + g);
        }
        double *ghb = R.gh + (size_t)b * R.mc;
        out(ghb + i, gP);
        out(ghb + nb + i, gQ);
        out(ghb + 2 * nb + 2 * N.nl + i, V2);
    }
    if (JP) {
        const double tG = twice(Gs), tB = twice(Bs);
        JP[nlow] = fma(tG, ei, pe);
        JP[k + nlow] = fma(tG, fi, pf);
        JQ[nlow] = fma(-tB, ei, qe);
        JQ[k + nlow] = fma(-tB, fi, qf);
        for (int q = 0; q < g1 - g0; q++) {
            const double v = gen_on(gm, gm ? __ldg(N.gen_ord + g0 + q) : 0) ? -1.0 : 0.0;
            JP[2 * k + q] = v;
            JQ[2 * k + q] = v;
        }
        double *Jv = Jb + N.nnzJ + 2 * (size_t)i;              // voltage row: 2 e_i, 2 f_i
        out(Jv, twice(ei));
        out(Jv + 1, twice(fi));
    }
    if (HM) {
        const double *lb = R.lam + (size_t)b * R.mc;
        const double lP = __ldg(lb + i), lQ = __ldg(lb + nb + i);
        const double muV = __ldg(lb + 2 * nb + 2 * N.nl + i);
        const double dsh = fma(lP, twice(Gs), fma(-lQ, twice(Bs), twice(muV)));
        HA[nlow] = hee + dsh;                                  // (e_i, e_i)
        HM[nlow] = hfe;                                        // (f_i, e_i)
        HM[k + nlow] = hff + dsh;                              // (f_i, f_i)
        if (g1 > g0) {
            const double sw = R.sigma * (R.obj_weight ? __ldg(R.obj_weight + b) : 1.0);
            for (int q = g0; q < g1; q++) {
                const int g = __ldg(N.gen_ord + q);
                out(Hb + N.hpg + g, gen_on(gm, g) ? sw * __ldg(N.c2g + g) : 0.0);
            }
        }
    }
    if (R.grad) {
        double *gb = R.grad + (size_t)b * N.n;
        out(gb + i, 0.0);
        out(gb + nb + i, 0.0);
        const double w = R.obj_weight ? __ldg(R.obj_weight + b) : 1.0;
        for (int q = g0; q < g1; q++) {
            const int g = __ldg(N.gen_ord + q);
            out(gb + 2 * nb + g, gen_on(gm, g) ? w * fma(__ldg(N.c2g + g), __ldg(xb + 2 * nb + g),
                                                         __ldg(N.c1g + g))
                                               : 0.0);
            out(gb + 2 * nb + ng + g, 0.0);
        }
    }
}

__global__ void __launch_bounds__(128) k_cart_bus(const DevNet N, const CartReq R, int nB) {
    const int per = (N.nb + 127) / 128;
    for (int it = blockIdx.x; it < nB * per; it += gridDim.x) {
        const int bl = it / per;
        const int i = (it - bl * per) * 128 + threadIdx.x;
        if (i < N.nb)
            cart_bus_item_at(N, R, R.b0 + bl, R.scratch + (size_t)bl * N.nslot * CNC, i,
                             cart_rows(N, R, R.b0 + bl, i));
    }
}

// The bus items of buses [i0, i0 + 128) of state b, by the whole block.  Thread r takes the
// tile's r-th bus by descending degree (the plan's permutation for 128-bus tiles, which maps every
// tile onto itself), so that a warp's slot walks have similar lengths.  When the tile's four row
// segments (J rows P and Q, H rows e and f: contiguous, the same layout as the polar rows) fit
// `cap` doubles of shared memory, the rows are assembled there and copied out with coalesced
// stores; otherwise they go straight to global memory.  Contains __syncthreads(): call from every
// thread of the block.
__device__ __forceinline__ void cart_bus_tile(const DevNet &N, const CartReq &R, int b, int i0,
                                              const double *scr, double *stage, int cap) {
    const int nb = N.nb, r = threadIdx.x;
    const int i1 = min(i0 + 128, nb);
    const int *perm = N.bus_perm + (size_t)stage_index(128) * nb;
    const int i = i0 + r < i1 ? __ldg(perm + i0 + r) : nb;
    const bool WJ = R.jval != nullptr, WH = R.hval != nullptr;
    const int p0 = row_start(N.bus_jP, i0, nb, N.jP_end), p1 = row_start(N.bus_jP, i1, nb, N.jP_end);
    const int q0 = row_start(N.bus_jQ, i0, nb, N.jQ_end);
    const int a0 = row_start(N.bus_hA, i0, nb, N.hA_end), a1 = row_start(N.bus_hA, i1, nb, N.hA_end);
    const int m0 = row_start(N.bus_hM, i0, nb, N.hM_end), m1 = row_start(N.bus_hM, i1, nb, N.hM_end);
    const int LP = WJ ? p1 - p0 : 0, LA = WH ? a1 - a0 : 0, LM = WH ? m1 - m0 : 0;
    const bool staged = (WJ || WH) && 2 * LP + LA + LM <= cap;
    if (i < i1) {
        BusRows W = cart_rows(N, R, b, i);
        if (staged) {
            if (WJ) {
                W.JP = stage + (__ldg(N.bus_jP + i) - p0);
                W.JQ = stage + LP + (__ldg(N.bus_jQ + i) - q0);
            }
            if (WH) {
                W.HA = stage + 2 * LP + (__ldg(N.bus_hA + i) - a0);
                W.HM = stage + 2 * LP + LA + (__ldg(N.bus_hM + i) - m0);
            }
        }
        cart_bus_item_at(N, R, b, scr, i, W);
    }
    if (staged) {
        __syncthreads();
        double *Jb = WJ ? R.jval + (size_t)b * R.nnzJc : nullptr;
        double *Hb = WH ? R.hval + (size_t)b * N.nnzH : nullptr;
        for (int e = r; e < LP; e += 128) {
            out(Jb + p0 + e, stage[e]);
            out(Jb + q0 + e, stage[LP + e]);
        }
        for (int e = r; e < LA; e += 128) out(Hb + a0 + e, stage[2 * LP + e]);
        for (int e = r; e < LM; e += 128) out(Hb + m0 + e, stage[2 * LP + LA + e]);
        __syncthreads();   // the next tile overwrites the stage
    }
}

// Objective of each state (the polar model's: it depends on Pg only).
__global__ void __launch_bounds__(OBJ_LANES) k_cart_obj(const DevNet N, const EvalReq R, int b0) {
    __shared__ double part[OBJ_LANES];
    obj_block<true, OBJ_LANES>(N, R, b0 + blockIdx.x, part);
}

// Persistent schedule of the cartesian evaluation: the polar model's ticketed work list
// (PersistParams, decode_item) over (state, 128 branches) and (state, 128 buses) items.  A branch
// item writes its branches' records into ring slot b mod ring once the bus items of state
// b - ring have consumed that slot (the last branch item first computes the state's objective); a bus
// item waits for all branch items of its state, assembles its buses' rows, discards the consumed
// records from L2 and signals.  Each item computes exactly what the chunked kernels compute for it, so both
// schedules give bitwise equal results.  Waits are bounded as in the polar kernel.
// MINB: resident CTAs per SM the register allocation must allow (1: the compiler's choice).
template <bool PS, int MINB>
__global__ void __launch_bounds__(128, MINB) k_cart_persist(const DevNet N, const CartReq R,
                                                      const PersistParams P) {
    __shared__ int s_item, s_ok;
    __shared__ double s_part[OBJ_LANES];
    extern __shared__ double stage[];
    int *done_br = P.ctr + 1, *done_bu = P.ctr + 1 + P.B;
    const size_t slot_doubles = (size_t)CNC * N.nslot;
    int next = 0;
    if (threadIdx.x == 0) next = atomicAdd(P.ctr, 1);
    for (;;) {
        if (threadIdx.x == 0) {
            s_item = next;
            if (next < P.total) next = atomicAdd(P.ctr, 1);
        }
        __syncthreads();
        const int t = s_item;
        if (t >= P.total) return;
        bool is_branch;
        int b, tile;
        decode_item(P, t, &is_branch, &b, &tile);
        double *scr = R.scratch + (size_t)(b % P.ring) * slot_doubles;
        // the objective reads x only: the state's last branch item computes it first (bus item
        // 0 when the net has no branches)
        if (R.f && is_branch == (P.Tbr > 0) && tile == (P.Tbr > 0 ? P.Tbr - 1 : 0)) {
            EvalReq E{};
            E.B = R.B;
            E.x = R.x; E.obj_weight = R.obj_weight; E.f = R.f; E.gen_mask = R.gen_mask;
            obj_block<true, 128>(N, E, b, s_part);
        }
        if (is_branch) {
            if (threadIdx.x == 0)
                s_ok = b < P.ring || bounded_wait(done_bu + (b - P.ring), P.Tbu, P.spin_limit,
                                                  N.status, ST_TIMEOUT_RING);
            __syncthreads();
            const int l = tile * 128 + threadIdx.x;
            if (s_ok && l < N.nl) cart_branch_item_at<PS>(N, R, b, scr, l);
            __syncthreads();
            if (threadIdx.x == 0) red_release_add(done_br + b);
        } else {
            if (threadIdx.x == 0)
                s_ok = bounded_wait(done_br + b, P.Tbr + P.force_timeout, P.spin_limit, N.status,
                                    ST_TIMEOUT_BUS);
            __syncthreads();
            if (s_ok) cart_bus_tile(N, R, b, tile * 128, scr, stage, R.stage_cap);
            __syncthreads();
            if (threadIdx.x < 32) {
                if (s_ok) {   // this item's records are consumed
                    const int i1 = min(N.nb, (tile + 1) * 128);
                    discard_lines(scr + (size_t)__ldg(N.slot_ptr + tile * 128) * CNC,
                                  scr + (size_t)__ldg(N.slot_ptr + i1) * CNC, threadIdx.x);
                    __syncwarp();   // the lanes' discards before lane 0's release
                }
                if (threadIdx.x == 0) red_release_add(done_bu + b);
            }
        }
    }
}

// ---- adjoint products of the cartesian constraint map c = [g; h] ----
//   JVP  out [B][m_c] = J u,  JTV  out [B][n] = J^T v,  HVP  out [B][n] = (grad^2 L) u.
// Each branch writes two values per end -- its P and Q row entries (JVP), or its contributions
// to the end bus's e and f components (JTV, HVP) -- ordered by branch; the bus kernel sums its
// slots' values in slot order and adds the shunt, voltage-row and generator terms.
enum CartAdjMode : int { CADJ_JVP = 0, CADJ_JTV = 1, CADJ_HVP = 2 };

struct CartAdjReq {
    int b0, mc;
    const double *x, *lam;
    const uint8_t *mask, *gen_mask;
    const double *obj_weight;
    double sigma;
    const double *v;            // JVP / HVP: [B][n]; JTV: [B][m_c]
    double *out;                // JVP: [B][m_c]; JTV / HVP: [B][n]
    double *scratch;            // [chunk][nl][4]
};

template <int MODE, bool PS>
__global__ void __launch_bounds__(128) k_cart_adj_branch(const DevNet N, const CartAdjReq A) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= N.nl) return;
    const int bl = blockIdx.y, b = A.b0 + bl;
    const int nb = N.nb, nl = N.nl;
    double *rf = A.scratch + ((size_t)bl * nl + l) * 4, *rt = rf + 2;
    const int fb = __ldg(N.f + l), tb = __ldg(N.t + l);
    const bool on = A.mask == nullptr || A.mask[(size_t)b * nl + l] != 0;
    if (!on) {
        put2c(rf, 0, 0.0, 0.0);
        put2c(rt, 0, 0.0, 0.0);
        if (MODE == CADJ_JVP) {
            A.out[(size_t)b * A.mc + 2 * nb + l] = 0.0;
            A.out[(size_t)b * A.mc + 2 * nb + nl + l] = 0.0;
        }
        return;
    }
    const double *xb = A.x + (size_t)b * N.n;
    const CartY y = cart_y<PS>(N, l);
    const CartBranch c = cart_terms<PS>(y, __ldg(xb + fb), __ldg(xb + nb + fb), __ldg(xb + tb),
                                        __ldg(xb + nb + tb));
    if (MODE == CADJ_JTV) {
        const double *vb = A.v + (size_t)b * A.mc;
        const double vhf2 = twice(__ldg(vb + 2 * nb + l)), vht2 = twice(__ldg(vb + 2 * nb + nl + l));
        // weights of grad P and grad Q at each end: row multiplier + 2 v_h (P or Q)
        const double wPf = fma(vhf2, c.Pf, __ldg(vb + fb)), wQf = fma(vhf2, c.Qf, __ldg(vb + nb + fb));
        const double wPt = fma(vht2, c.Pt, __ldg(vb + tb)), wQt = fma(vht2, c.Qt, __ldg(vb + nb + tb));
        put2c(rf, 0, fma(wPf, c.p1f, fma(wQf, c.q1f, fma(wPt, c.p3t, wQt * c.p4t))),
              fma(wPf, c.p2f, fma(wQf, c.q2f, fma(wPt, c.p4t, -(wQt * c.p3t)))));
        put2c(rt, 0, fma(wPt, c.p1t, fma(wQt, c.q1t, fma(wPf, c.p3f, wQf * c.p4f))),
              fma(wPt, c.p2t, fma(wQt, c.q2t, fma(wPf, c.p4f, -(wQf * c.p3f)))));
        return;
    }
    const double *ub = A.v + (size_t)b * N.n;
    const double uef = __ldg(ub + fb), uff = __ldg(ub + nb + fb);
    const double uet = __ldg(ub + tb), uft = __ldg(ub + nb + tb);
    if (MODE == CADJ_JVP) {
        const double dPf = fma(c.p1f, uef, fma(c.p2f, uff, fma(c.p3f, uet, c.p4f * uft)));
        const double dQf = fma(c.q1f, uef, fma(c.q2f, uff, fma(c.p4f, uet, -(c.p3f * uft))));
        const double dPt = fma(c.p1t, uet, fma(c.p2t, uft, fma(c.p3t, uef, c.p4t * uff)));
        const double dQt = fma(c.q1t, uet, fma(c.q2t, uft, fma(c.p4t, uef, -(c.p3t * uff))));
        put2c(rf, 0, dPf, dQf);
        put2c(rt, 0, dPt, dQt);
        double *ob = A.out + (size_t)b * A.mc;
        ob[2 * nb + l] = twice(fma(c.Pf, dPf, c.Qf * dQf));
        ob[2 * nb + nl + l] = twice(fma(c.Pt, dPt, c.Qt * dQt));
    } else {
        const double *lb = A.lam + (size_t)b * A.mc;
        const CartHess h = cart_hess<PS>(y, c, __ldg(lb + fb), __ldg(lb + nb + fb), __ldg(lb + tb),
                                         __ldg(lb + nb + tb), __ldg(lb + 2 * nb + l),
                                         __ldg(lb + 2 * nb + nl + l));
        // rows of the block over (e_f, f_f, e_t, f_t) times u
        put2c(rf, 0, fma(h.eef, uef, fma(h.fef, uff, fma(h.eeft, uet, h.ef_ft * uft))),
              fma(h.fef, uef, fma(h.fff, uff, fma(h.ff_et, uet, h.ffft * uft))));
        put2c(rt, 0, fma(h.eeft, uef, fma(h.ff_et, uff, fma(h.eet, uet, h.fet * uft))),
              fma(h.ef_ft, uef, fma(h.ffft, uff, fma(h.fet, uet, h.fft * uft))));
    }
}

template <int MODE>
__global__ void __launch_bounds__(128) k_cart_adj_bus(const DevNet N, const CartAdjReq A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N.nb) return;
    const int bl = blockIdx.y, b = A.b0 + bl;
    const int nb = N.nb, ng = N.ng, nl = N.nl;
    const double *scr = A.scratch + (size_t)bl * nl * 4;
    const int s0 = __ldg(N.slot_ptr + i), s1 = __ldg(N.slot_ptr + i + 1);
    const int g0 = __ldg(N.gen_ptr + i), g1 = __ldg(N.gen_ptr + i + 1);
    double s0v = 0.0, s1v = 0.0;
    for (int s = s0; s < s1; s++) {
        const double2 r = ld2(scr + 2 * (size_t)__ldg(N.slot_ref + s));
        s0v += r.x;
        s1v += r.y;
    }
    const double *xb = A.x + (size_t)b * N.n;
    const double ei = __ldg(xb + i), fi = __ldg(xb + nb + i);
    const double Gs = __ldg(N.Gs + i), Bs = __ldg(N.Bs + i);
    const uint8_t *gm = A.gen_mask && g1 > g0 ? A.gen_mask + (size_t)b * ng : nullptr;
    if (MODE == CADJ_JVP) {
        const double *ub = A.v + (size_t)b * N.n;
        const double dV = twice(fma(ei, __ldg(ub + i), fi * __ldg(ub + nb + i)));   // d(e^2 + f^2)
        double oP = fma(Gs, dV, s0v), oQ = fma(-Bs, dV, s1v);
        for (int q = g0; q < g1; q++) {
            const int g = __ldg(N.gen_ord + q);
            if (!gen_on(gm, g)) continue;
            oP -= __ldg(ub + 2 * nb + g);
            oQ -= __ldg(ub + 2 * nb + ng + g);
        }
        double *ob = A.out + (size_t)b * A.mc;
        ob[i] = oP;
        ob[nb + i] = oQ;
        ob[2 * nb + 2 * nl + i] = dV;
    } else if (MODE == CADJ_JTV) {
        const double *vb = A.v + (size_t)b * A.mc;
        const double vP = __ldg(vb + i), vQ = __ldg(vb + nb + i);
        const double coef = twice(fma(Gs, vP, fma(-Bs, vQ, __ldg(vb + 2 * nb + 2 * nl + i))));
        double *ob = A.out + (size_t)b * N.n;
        ob[i] = fma(coef, ei, s0v);
        ob[nb + i] = fma(coef, fi, s1v);
        for (int q = g0; q < g1; q++) {
            const int g = __ldg(N.gen_ord + q);
            ob[2 * nb + g] = gen_on(gm, g) ? dneg(vP) : 0.0;
            ob[2 * nb + ng + g] = gen_on(gm, g) ? dneg(vQ) : 0.0;
        }
    } else {
        const double *lb = A.lam + (size_t)b * A.mc;
        const double *ub = A.v + (size_t)b * N.n;
        const double dsh = twice(fma(__ldg(lb + i), Gs,
                                     fma(-__ldg(lb + nb + i), Bs, __ldg(lb + 2 * nb + 2 * nl + i))));
        double *ob = A.out + (size_t)b * N.n;
        ob[i] = fma(dsh, __ldg(ub + i), s0v);
        ob[nb + i] = fma(dsh, __ldg(ub + nb + i), s1v);
        const double sw = A.sigma * (A.obj_weight ? __ldg(A.obj_weight + b) : 1.0);
        for (int q = g0; q < g1; q++) {
            const int g = __ldg(N.gen_ord + q);
            ob[2 * nb + g] = gen_on(gm, g) ? sw * __ldg(N.c2g + g) * __ldg(ub + 2 * nb + g) : 0.0;
            ob[2 * nb + ng + g] = 0.0;
        }
    }
}

size_t record_bytes(const DevNet &N) { return (size_t)N.nslot * CNC * sizeof(double); }

// Resident CTAs of a kernel on the current device (looked up once per device and kernel).
int resident_ctas(const void *kernel, int slot) {
    static std::atomic<int> cache[64][3];   // slots: branch, bus, branch with phase shifters
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    int v = cache[dev][slot].load(std::memory_order_relaxed);
    if (v == 0) {
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 128, 0) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            per_sm < 1 || sms < 1) {
            cudaGetLastError();
            return 152;
        }
        v = per_sm * sms;
        cache[dev][slot].store(v, std::memory_order_relaxed);
    }
    return v;
}

int chunk_states(const DevNet &N, int B) {
    const size_t per = std::max<size_t>(record_bytes(N), 1);
    return (int)std::max<size_t>(1, std::min<size_t>((size_t)std::min(B, 65535), kChunkRecordBytes / per));
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// Workspace of the chunked schedule for B states: `ring` chunks of records.
size_t chunked_bytes(const DevNet &N, int B) {
    const int chunk = chunk_states(N, B);
    const int ring = std::min(kRing, (B + chunk - 1) / chunk);
    return (size_t)ring * chunk * record_bytes(N);
}

// Ring slots of the persistent schedule are sized to stay in L2 with room to spare.
constexpr size_t kPersistRingBytes = (size_t)64 << 20;

// Shared memory of a persistent bus tile (the largest 128-bus tile's row segments, within the
// budget that keeps the register-limited number of resident CTAs per SM) and the resident CTAs
// of the persistent kernel with it, looked up once per device, variant and need.
struct CartShape {
    int cap, grid;
};

// Resident CTAs of 128 threads per SM that the persistent kernel's registers must allow for a
// target of occ resident warps (exago_config.occupancy: 16, the default, or 24; 8: the
// compiler's choice).  Measured on the 2,000-bus grid x 512 states with staged rows: 0.487 ms at
// 16 (103 registers) and at 8 (105), 0.62 ms at 24 (80 registers, spills); with rows straight to
// memory 0.50-0.52 ms at every setting.
constexpr int cart_minb(int occ) { return occ == 8 ? 1 : occ / 4; }

template <int OCC>
const void *cart_persist_fn_occ(bool ps) {
    return ps ? (const void *)k_cart_persist<true, cart_minb(OCC)>
              : (const void *)k_cart_persist<false, cart_minb(OCC)>;
}

const void *cart_persist_fn(bool ps, int occ) {
    switch (occ) {
        case 8: return cart_persist_fn_occ<8>(ps);
        case 16: return cart_persist_fn_occ<16>(ps);
        case 24: return cart_persist_fn_occ<24>(ps);
        default: return cart_persist_fn_occ<16>(ps);
    }
}

template <int OCC>
void launch_cart_persist(bool ps, int grid, size_t smem, cudaStream_t st, const DevNet &N,
                         const CartReq &R, const PersistParams &P) {
    if (ps) k_cart_persist<true, cart_minb(OCC)><<<grid, 128, smem, st>>>(N, R, P);
    else k_cart_persist<false, cart_minb(OCC)><<<grid, 128, smem, st>>>(N, R, P);
}

CartShape cart_shape(const DevNet &N, int occ) {
    const bool ps = N.Gtf != nullptr;
    const int want = std::max(0, N.stage_cap_rows[stage_index(128)]);
    CartShape sh{0, 152};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return sh;
    }
    static std::mutex mu;
    static std::map<uint64_t, CartShape> cache;
    const uint64_t key = ((uint64_t)dev << 48) | ((uint64_t)occ << 40) | ((uint64_t)ps << 32) |
                         (uint64_t)(uint32_t)want;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    const void *k = cart_persist_fn(ps, occ);
    int sms = 0, smem_sm = 0, by_regs = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&by_regs, k, 128, 0) != cudaSuccess ||
        by_regs < 1 || sms < 1) {
        cudaGetLastError();
        return sh;
    }
    const long budget = ((long)smem_sm / by_regs - 4096) / 8;
    sh.cap = (int)(std::max<long>(0, std::min<long>(want, budget)) & ~1l);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 128, (size_t)sh.cap * sizeof(double)) !=
            cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    sh.grid = per_sm * sms;
    cache[key] = sh;
    return sh;
}

// Launch settings of the persistent schedule for B >= 1 states, from the net's configuration.
struct CartPersist {
    int grid, cap, occ, lag, ring;
    long long spin_limit;
    int force_timeout;
    bool use_graph;
};

bool cart_is_persistent(const exago_config &c) {
    return c.schedule != EXAGO_SCHED_KERNELS && c.schedule != EXAGO_SCHED_PIPELINED;
}

CartPersist cart_persist_plan(const exago_config &c, const DevNet &N, int B) {
    CartPersist p{};
    p.occ = c.occupancy == 8 || c.occupancy == 24 ? c.occupancy : 16;
    const CartShape sh = cart_shape(N, p.occ);
    p.grid = sh.grid;
    // rows through shared memory unless EXAGO_STAGE_OFF asks for direct stores
    p.cap = c.stage_records == EXAGO_STAGE_OFF ? 0 : sh.cap;
    // bus items trail branch items by 4/3 of the states the resident CTAs hold in branch work,
    // plus two (the polar schedule's rule); the ring holds up to three lags within its L2 budget
    const int Tbr = (N.nl + 127) / 128;
    int lag = c.lag > 0 ? c.lag : (Tbr > 0 ? (4 * p.grid + 3 * Tbr - 1) / (3 * Tbr) : 1) + 2;
    lag = std::max(1, std::min(lag, B));
    const int fit = (int)std::min<size_t>(1 << 20, kPersistRingBytes / std::max<size_t>(record_bytes(N), 1));
    int ring = c.ring > 0 ? c.ring : std::max(lag + 2, std::min(3 * lag + 2, fit));
    if (ring <= lag) ring = lag + 1;
    if (ring > B + 1) ring = B + 1;
    p.lag = lag;
    p.ring = ring;
    p.spin_limit = c.spin_limit > 0 ? c.spin_limit : (1ll << 22);
    p.force_timeout = c.test_force_timeout ? 1 : 0;
    p.use_graph = c.use_graph != EXAGO_GRAPH_OFF;
    return p;
}

size_t counter_bytes(int B) { return round256((size_t)(1 + 2 * (size_t)B) * sizeof(int)); }

size_t persist_bytes(const DevNet &N, const CartPersist &p, int B) {
    return round256((size_t)p.ring * record_bytes(N)) + counter_bytes(B);
}

// One adjoint product over the batch, in chunks of states whose branch values fit the workspace.
exago_status cart_adjoint(exago_net_t net, const exago_batch *bt, const double *in, double *out,
                          int mode) {
    const HostPlan *plan = nullptr;
    const DevNet *dev = nullptr;
    int device = -1;
    if (!net_internal_view(net, &plan, &dev, &device))
        return set_last_error(net ? EXAGO_ESTATE : EXAGO_EINVAL,
                              net ? "net was planned without a device" : "net is NULL");
    if (!bt) return set_last_error(EXAGO_EINVAL, "batch is NULL");
    if (bt->B < 0) return set_last_error(EXAGO_EINVAL, "batch B < 0");
    if (bt->B == 0) return EXAGO_OK;
    if (!bt->x) return set_last_error(EXAGO_EINVAL, "batch x is NULL");
    if (!in || !out) return set_last_error(EXAGO_EINVAL, "input or output vector is NULL");
    if (mode == CADJ_HVP && !bt->lambda)
        return set_last_error(EXAGO_EINVAL, "batch lambda is NULL (needed by the Hessian)");
    const DevNet &N = *dev;
    const size_t per = (size_t)std::max(N.nl, 1) * 4 * sizeof(double);
    int chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)std::min(bt->B, 65535),
                                                          kAdjChunkBytes / per));
    void *ws = bt->workspace;
    if (ws) {
        if (((uintptr_t)ws & 255) != 0)
            return set_last_error(EXAGO_EINVAL, "workspace not 256-byte aligned");
        if (bt->workspace_bytes < per)
            return set_last_error(EXAGO_EINVAL, "workspace smaller than one state's branch values");
        chunk = (int)std::min<size_t>((size_t)chunk, bt->workspace_bytes / per);
    }
    cudaStream_t st = (cudaStream_t)bt->stream;
    // the net's lock stays held until every kernel that uses its workspace is queued
    return with_net_workspace(net, ws, (size_t)chunk * per, st, false,
                              [&](void *w, const PipeLaunch *) -> exago_status {
        CartAdjReq A{};
        A.mc = N.m + N.nb;
        A.x = bt->x; A.lam = bt->lambda; A.mask = bt->mask; A.gen_mask = bt->gen_mask;
        A.obj_weight = bt->obj_weight; A.sigma = bt->obj_factor;
        A.v = in; A.out = out;
        A.scratch = (double *)w;
        for (int b0 = 0; b0 < bt->B; b0 += chunk) {
            const int nB = std::min(chunk, bt->B - b0);
            A.b0 = b0;
            const dim3 gbr((N.nl + 127) / 128, nB), gbu((N.nb + 127) / 128, nB);
            const bool ps = N.Gtf != nullptr;   // phase-shifting transformers
            if (mode == CADJ_JVP) {
                if (N.nl > 0 && ps) k_cart_adj_branch<CADJ_JVP, true><<<gbr, 128, 0, st>>>(N, A);
                else if (N.nl > 0) k_cart_adj_branch<CADJ_JVP, false><<<gbr, 128, 0, st>>>(N, A);
                k_cart_adj_bus<CADJ_JVP><<<gbu, 128, 0, st>>>(N, A);
            } else if (mode == CADJ_JTV) {
                if (N.nl > 0 && ps) k_cart_adj_branch<CADJ_JTV, true><<<gbr, 128, 0, st>>>(N, A);
                else if (N.nl > 0) k_cart_adj_branch<CADJ_JTV, false><<<gbr, 128, 0, st>>>(N, A);
                k_cart_adj_bus<CADJ_JTV><<<gbu, 128, 0, st>>>(N, A);
            } else {
                if (N.nl > 0 && ps) k_cart_adj_branch<CADJ_HVP, true><<<gbr, 128, 0, st>>>(N, A);
                else if (N.nl > 0) k_cart_adj_branch<CADJ_HVP, false><<<gbr, 128, 0, st>>>(N, A);
                k_cart_adj_bus<CADJ_HVP><<<gbu, 128, 0, st>>>(N, A);
            }
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return set_last_error(EXAGO_ECUDA, std::string("cartesian adjoint launch: ") +
                                                   cudaGetErrorString(e));
        return EXAGO_OK;
    });
}

// The persistent schedule of one call (rows wanted, nb > 0): the counters' memset and one launch,
// through the net's graph cache when allowed.
exago_status cart_eval_persistent(exago_net_t net, const DevNet &N, const exago_batch *bt, CartReq R,
                                  const exago_config &cfg, bool allow_graph) {
    const int B = bt->B;
    CartPersist p = cart_persist_plan(cfg, N, B);
    const size_t slot = record_bytes(N);
    void *ws = bt->workspace;
    if (ws) {   // a smaller caller workspace takes fewer ring slots (at least two)
        if (((uintptr_t)ws & 255) != 0)
            return set_last_error(EXAGO_EINVAL, "workspace not 256-byte aligned");
        const size_t cb = counter_bytes(B), have = bt->workspace_bytes;
        size_t fit = have > cb ? (have - cb) / std::max<size_t>(slot, 1) : 0;
        while (fit > 0 && round256(fit * slot) + cb > have) fit--;
        if (fit < 2)
            return set_last_error(EXAGO_EINVAL, "workspace smaller than exago_eval_cart_workspace_size");
        if ((size_t)p.ring > fit) {
            p.ring = (int)fit;
            if (p.lag >= p.ring) p.lag = p.ring - 1;
        }
    }
    cudaStream_t st = (cudaStream_t)bt->stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(st, &cap);
    if (ce != cudaSuccess)
        return set_last_error(EXAGO_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(ce));
    const bool graph = allow_graph && p.use_graph && cap == cudaStreamCaptureStatusNone;
    const bool ps = N.Gtf != nullptr;   // phase-shifting transformers
    PersistParams P{};
    P.B = B;
    P.group = 1;
    P.Tbr = (N.nl + 127) / 128;
    P.Tbu = (N.nb + 127) / 128;
    P.lag = p.lag;
    P.ring = p.ring;
    P.total = B * (P.Tbr + P.Tbu);
    P.spin_limit = p.spin_limit;
    P.force_timeout = p.force_timeout;
    P.times = nullptr;
    const int grid = std::min(p.grid, P.total);
    R.stage_cap = p.cap;
    // the net's lock stays held until the launch (or the graph launch) is queued
    return with_net_workspace(net, ws, persist_bytes(N, p, B), st, false,
                              [&](void *w, const PipeLaunch *) -> exago_status {
        R.scratch = (double *)w;
        P.ctr = (int *)((char *)w + round256((size_t)p.ring * slot));
        auto launch = [&](cudaStream_t cs) -> int {
            cudaError_t e = cudaMemsetAsync(P.ctr, 0, (size_t)(1 + 2 * (size_t)B) * sizeof(int), cs);
            if (e != cudaSuccess) return (int)e;
            const size_t smem = (size_t)R.stage_cap * sizeof(double);
            switch (p.occ) {
                case 8: launch_cart_persist<8>(ps, grid, smem, cs, N, R, P); break;
                case 24: launch_cart_persist<24>(ps, grid, smem, cs, N, R, P); break;
                default: launch_cart_persist<16>(ps, grid, smem, cs, N, R, P); break;
            }
            return (int)cudaGetLastError();
        };
        if (graph) {
            uint64_t sg;
            std::memcpy(&sg, &R.sigma, sizeof sg);
            const std::vector<uint64_t> key = {
                0xCA470u + (uint64_t)ps, (uint64_t)R.x, (uint64_t)R.lam, (uint64_t)R.mask,
                (uint64_t)R.gen_mask, (uint64_t)R.pd_scale, (uint64_t)R.obj_weight, sg,
                (uint64_t)R.f, (uint64_t)R.grad, (uint64_t)R.gh, (uint64_t)R.jval, (uint64_t)R.hval,
                (uint64_t)R.scratch, (uint64_t)P.ctr, (uint64_t)B, (uint64_t)grid, (uint64_t)P.lag,
                (uint64_t)P.ring, (uint64_t)P.spin_limit, (uint64_t)P.force_timeout,
                (uint64_t)R.stage_cap, (uint64_t)p.occ};
            return net_graph_launch_locked(net, key, launch, st);
        }
        const int e = launch(st);
        if (e != 0)
            return set_last_error(EXAGO_ECUDA, std::string("cartesian persistent launch: ") +
                                                   cudaGetErrorString((cudaError_t)e));
        return EXAGO_OK;
    });
}

// One cartesian evaluation call: the persistent schedule by default, the chunked two-stream
// schedule when the net's configuration asks for EXAGO_SCHED_PIPELINED or EXAGO_SCHED_KERNELS.
exago_status cart_eval(exago_net_t net, const exago_batch *bt, double *f, double *grad, double *gh,
                       double *jval, double *hval, bool allow_graph) {
    const HostPlan *plan = nullptr;
    const DevNet *dev = nullptr;
    int device = -1;
    if (!net_internal_view(net, &plan, &dev, &device))
        return set_last_error(net ? EXAGO_ESTATE : EXAGO_EINVAL,
                              net ? "net was planned without a device" : "net is NULL");
    if (!bt) return set_last_error(EXAGO_EINVAL, "batch is NULL");
    if (bt->B < 0) return set_last_error(EXAGO_EINVAL, "batch B < 0");
    if (bt->B == 0) return EXAGO_OK;
    if (!bt->x) return set_last_error(EXAGO_EINVAL, "batch x is NULL");
    if (hval && !bt->lambda)
        return set_last_error(EXAGO_EINVAL, "batch lambda is NULL (needed by the Hessian)");
    const DevNet &N = *dev;
    cudaStream_t st = (cudaStream_t)bt->stream;
    const bool rows = gh || jval || hval || grad;
    const exago_config cfg = net_config(net);
    const bool persistent = rows && N.nb > 0 && cart_is_persistent(cfg);
    if (persistent) {
        CartReq R{};
        R.B = bt->B;
        R.mc = N.m + N.nb;
        R.nnzJc = N.nnzJ + 2 * (int64_t)N.nb;
        R.x = bt->x; R.lam = bt->lambda; R.mask = bt->mask; R.gen_mask = bt->gen_mask;
        R.pd_scale = bt->pd_scale; R.obj_weight = bt->obj_weight; R.sigma = bt->obj_factor;
        R.f = f; R.grad = grad; R.gh = gh; R.jval = jval; R.hval = hval;
        exago_status s = cart_eval_persistent(net, N, bt, R, cfg, allow_graph);
        if (s != EXAGO_OK) return s;
    } else {
        if (rows && N.nb > 0) {
            const int chunk = chunk_states(N, bt->B);
            const size_t chunk_bytes = (size_t)chunk * record_bytes(N);
            const int nchunks = (bt->B + chunk - 1) / chunk;
            int ring = std::min(kRing, nchunks);
            void *ws = bt->workspace;
            if (ws) {
                if (((uintptr_t)ws & 255) != 0)
                    return set_last_error(EXAGO_EINVAL, "workspace not 256-byte aligned");
                if (bt->workspace_bytes < chunk_bytes)
                    return set_last_error(EXAGO_EINVAL, "workspace smaller than exago_eval_cart_workspace_size");
                ring = (int)std::min<size_t>((size_t)ring, bt->workspace_bytes / std::max<size_t>(chunk_bytes, 1));
            }
            CartReq R{};
            R.B = bt->B;
            R.mc = N.m + N.nb;
            R.nnzJc = N.nnzJ + 2 * (int64_t)N.nb;
            R.x = bt->x; R.lam = bt->lambda; R.mask = bt->mask; R.gen_mask = bt->gen_mask;
            R.pd_scale = bt->pd_scale; R.obj_weight = bt->obj_weight; R.sigma = bt->obj_factor;
            R.f = f; R.grad = grad; R.gh = gh; R.jval = jval; R.hval = hval;
            const bool ps = N.Gtf != nullptr;   // phase-shifting transformers
            const void *kbr = ps ? (const void *)k_cart_branch<true> : (const void *)k_cart_branch<false>;
            const int br_ctas = resident_ctas(kbr, ps ? 2 : 0);
            const int bu_ctas = resident_ctas((const void *)k_cart_bus, 1);
            // chunk k: branch kernel on `main`, then its bus kernel on `side` (after an event), so the
            // FP64-bound branch work of chunk k + 1 overlaps the latency-bound bus work of chunk k;
            // the branch kernel of chunk k waits for the bus kernel of chunk k - ring, whose ring
            // slot it overwrites.  With one chunk or one ring slot everything runs on `main`.
            auto run = [&](void *ws, cudaStream_t main, cudaStream_t side, const PipeLaunch *pl) {
                if (pl) {
                    cudaEventRecord(pl->ev_fork, main);
                    cudaStreamWaitEvent(side, pl->ev_fork, 0);
                }
                for (int k = 0; k < nchunks; k++) {
                    const int b0 = k * chunk, nB = std::min(chunk, bt->B - b0);
                    CartReq Rk = R;
                    Rk.b0 = b0;
                    Rk.scratch = (double *)ws + (size_t)(k % ring) * chunk * N.nslot * CNC;
                    const int br_items = nB * ((N.nl + 127) / 128), bus_items = nB * ((N.nb + 127) / 128);
                    if (pl && k >= ring) cudaStreamWaitEvent(main, pl->ev_bu[(k - ring) % (ring + 1)], 0);
                    if (N.nl > 0)
                        if (ps) k_cart_branch<true><<<std::min(br_items, br_ctas), 128, 0, main>>>(N, Rk, nB);
                        else k_cart_branch<false><<<std::min(br_items, br_ctas), 128, 0, main>>>(N, Rk, nB);
                    cudaStream_t bs = main;
                    if (pl) {
                        cudaEventRecord(pl->ev_br[k % (ring + 1)], main);
                        cudaStreamWaitEvent(side, pl->ev_br[k % (ring + 1)], 0);
                        bs = side;
                    }
                    k_cart_bus<<<std::min(bus_items, bu_ctas), 128, 0, bs>>>(N, Rk, nB);
                    if (pl) cudaEventRecord(pl->ev_bu[k % (ring + 1)], side);
                }
                if (pl) {
                    cudaEventRecord(pl->ev_join, side);
                    cudaStreamWaitEvent(main, pl->ev_join, 0);
                }
                return EXAGO_OK;
            };
            // the net's lock stays held until every kernel that uses its workspace is queued
            const bool pipe = nchunks > 1 && ring > 1;
            exago_status s = with_net_workspace(
                net, ws, (size_t)ring * chunk_bytes, st, pipe,
                [&](void *w, const PipeLaunch *pl) {
                    return pl ? run(w, st, pl->side, pl) : run(w, st, st, nullptr);
                });
            if (s != EXAGO_OK) return s;
        }
    }
    if (f && !persistent) {
        EvalReq E{};
        E.B = bt->B;
        E.x = bt->x; E.obj_weight = bt->obj_weight; E.f = f; E.gen_mask = bt->gen_mask;
        for (int b0 = 0; b0 < bt->B; b0 += 65535)
            k_cart_obj<<<std::min(65535, bt->B - b0), OBJ_LANES, 0, st>>>(N, E, b0);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_last_error(EXAGO_ECUDA, std::string("cartesian evaluation launch: ") +
                                               cudaGetErrorString(e));
    return EXAGO_OK;
}

}  // namespace

int cart_allow_stage() {
    const int bytes = kStageMaxDoubles * (int)sizeof(double);
    cudaError_t e = cudaSuccess;
    for (int occ : {8, 16, 24})
        for (bool ps : {false, true})
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(cart_persist_fn(ps, occ),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return (int)e;
}

exago_status eval_cart_direct(exago_net_t net, const exago_batch *bt, double *f, double *grad,
                              double *gh, double *jval, double *hval) {
    return cart_eval(net, bt, f, grad, gh, jval, hval, false);
}

}  // namespace exago

using namespace exago;

extern "C" {

exago_status exago_net_dims_cart(exago_net_t net, int *n, int *m_eq, int *m_ineq, int64_t *nnzJ,
                                 int64_t *nnzH) {
    int nn = 0, me = 0, mi = 0;
    int64_t nj = 0, nh = 0;
    exago_status s = exago_net_dims(net, &nn, &me, &mi, &nj, &nh);
    if (s != EXAGO_OK) return s;
    const int nb = me / 2;
    if (n) *n = nn;
    if (m_eq) *m_eq = me;
    if (m_ineq) *m_ineq = mi + nb;
    if (nnzJ) *nnzJ = nj + 2 * (int64_t)nb;
    if (nnzH) *nnzH = nh;
    return EXAGO_OK;
}

exago_status exago_net_jac_pattern_cart(exago_net_t net, int64_t *rowptr, int *col) {
    int nn = 0, me = 0, mi = 0;
    int64_t nj = 0, nh = 0;
    exago_status s = exago_net_dims(net, &nn, &me, &mi, &nj, &nh);
    if (s != EXAGO_OK) return s;
    if (!rowptr || !col) return set_last_error(EXAGO_EINVAL, "null argument");
    if ((s = exago_net_jac_pattern(net, rowptr, col)) != EXAGO_OK) return s;
    const int nb = me / 2, m = me + mi;
    for (int i = 0; i < nb; i++) {   // voltage row i: columns e_i, f_i
        col[nj + 2 * i] = i;
        col[nj + 2 * i + 1] = nb + i;
        rowptr[m + i + 1] = nj + 2 * (int64_t)(i + 1);
    }
    return EXAGO_OK;
}

exago_status exago_eval_cart_workspace_size(exago_net_t net, int B, size_t *bytes) {
    const HostPlan *plan = nullptr;
    const DevNet *dev = nullptr;
    int device = -1;
    if (!bytes) return set_last_error(EXAGO_EINVAL, "bytes is NULL");
    if (!net_internal_view(net, &plan, &dev, &device))
        return set_last_error(net ? EXAGO_ESTATE : EXAGO_EINVAL,
                              net ? "net was planned without a device" : "net is NULL");
    if (B < 0) return set_last_error(EXAGO_EINVAL, "B < 0");
    if (B == 0) {
        *bytes = 0;
        return EXAGO_OK;
    }
    // enough for either schedule, so that a later change of the configuration keeps it valid
    const size_t p = persist_bytes(*dev, cart_persist_plan(net_config(net), *dev, B), B);
    *bytes = std::max(p, chunked_bytes(*dev, B));
    return EXAGO_OK;
}

exago_status exago_eval_cart(exago_net_t net, const exago_batch *bt, double *f, double *grad,
                             double *gh, double *jval, double *hval) {
    return cart_eval(net, bt, f, grad, gh, jval, hval, true);
}

exago_status exago_eval_cart_jvp(exago_net_t net, const exago_batch *batch, const double *u,
                                 double *out) {
    return cart_adjoint(net, batch, u, out, CADJ_JVP);
}

exago_status exago_eval_cart_jtv(exago_net_t net, const exago_batch *batch, const double *v,
                                 double *out) {
    return cart_adjoint(net, batch, v, out, CADJ_JTV);
}

exago_status exago_eval_cart_hvp(exago_net_t net, const exago_batch *batch, const double *u,
                                 double *out) {
    return cart_adjoint(net, batch, u, out, CADJ_HVP);
}

}  // extern "C"
