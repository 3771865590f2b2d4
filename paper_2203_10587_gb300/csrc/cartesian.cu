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
#include <string>

#include "eval_items.cuh"

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
};

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
// (Gt, Bt): P_t = Gtt s_t + Gt a - Bt bf, Q_t = -Btt s_t - Gt bf - Bt a, and the to end's
// admittance-voltage products below use Gt, Bt; without, one set of products serves both ends.
template <bool PS>
__device__ __forceinline__ CartBranch cart_terms(const CartY &y, double ef, double ff, double et,
                                                 double ft) {
    const double G = y.G, Bm = y.Bm, Gff = y.Gff, Bff = y.Bff, Gtt = y.Gtt, Btt = y.Btt;
    const double Gff2 = y.Gff2, Bff2 = y.Bff2, Gtt2 = y.Gtt2, Btt2 = y.Btt2;
    CartBranch c;
    // a = Vf Vt cos th, bf = Vf Vt sin th (th = Va_f - Va_t); the to end sees -bf
    const double a = fma(ef, et, ff * ft);
    const double bf = fma(ff, et, -(ef * ft));
    const double sf = fma(ef, ef, ff * ff), st = fma(et, et, ft * ft);
    const double Ga = G * a, Ba = Bm * a, Gb = G * bf, Bb = Bm * bf;
    c.Pf = fma(Gff, sf, Ga + Bb);
    c.Qf = fma(-Bff, sf, Gb - Ba);
    if (PS) {
        const double Gta = y.Gt * a, Bta = y.Bt * a, Gtb = y.Gt * bf, Btb = y.Bt * bf;
        c.Pt = fma(Gtt, st, Gta - Btb);
        c.Qt = fma(-Btt, st, -(Gtb + Bta));
    } else {
        c.Pt = fma(Gtt, st, Ga - Bb);
        c.Qt = fma(-Btt, st, -(Gb + Ba));
    }
    // admittance-voltage products shared by both ends' derivatives
    const double Gef = G * ef, Gff_ = G * ff, Get = G * et, Gft_ = G * ft;
    const double Bef = Bm * ef, Bff_ = Bm * ff, Bet = Bm * et, Bft_ = Bm * ft;
    const double u1 = Get - Bft_, u2 = Gft_ + Bet;
    c.p1f = fma(Gff2, ef, u1); c.p2f = fma(Gff2, ff, u2);
    c.q1f = fma(-Bff2, ef, -u2); c.q2f = fma(-Bff2, ff, u1);
    c.p3f = Gef + Bff_; c.p4f = Gff_ - Bef;
    double w1, w2;
    if (PS) {
        const double Gtef = y.Gt * ef, Gtff = y.Gt * ff, Gtet = y.Gt * et, Gtft = y.Gt * ft;
        const double Btef = y.Bt * ef, Btff = y.Bt * ff, Btet = y.Bt * et, Btft = y.Bt * ft;
        w1 = Gtef - Btff;
        w2 = Gtff + Btef;
        c.p3t = Gtet + Btft; c.p4t = Gtft - Btet;
    } else {
        w1 = Gef - Bff_;
        w2 = Gff_ + Bef;
        c.p3t = Get + Bft_; c.p4t = Gft_ - Bet;
    }
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

// One (state, branch) item of the branch kernel.
template <bool PS>
__device__ __forceinline__ void cart_branch_item(const DevNet &N, const CartReq &R, int bl, int l) {
    const int b = R.b0 + bl;
    const int nb = N.nb, nl = N.nl;
    double *scr = R.scratch + (size_t)bl * N.nslot * CNC;
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
        if (ghb) { ghb[2 * nb + l] = 0.0; ghb[2 * nb + nl + l] = 0.0; }
        if (Jf)
            for (int k = 0; k < 4; k++) { Jf[k] = 0.0; Jt[k] = 0.0; }
        return;
    }
    const double *xb = R.x + (size_t)b * N.n;
    const CartY y = cart_y<PS>(N, l);
    const CartBranch c = cart_terms<PS>(y, __ldg(xb + fb), __ldg(xb + nb + fb), __ldg(xb + tb),
                                        __ldg(xb + nb + tb));
    if (ghb) {
        ghb[2 * nb + l] = fma(c.Pf, c.Pf, c.Qf * c.Qf);
        ghb[2 * nb + nl + l] = fma(c.Pt, c.Pt, c.Qt * c.Qt);
    }
    if (Jf) {
        // grad |S|^2 = 2 P grad P + 2 Q grad Q, columns (e_lo, e_hi, f_lo, f_hi)
        const double Pf2 = twice(c.Pf), Qf2 = twice(c.Qf), Pt2 = twice(c.Pt), Qt2 = twice(c.Qt);
        const double hff_e = fma(Pf2, c.p1f, Qf2 * c.q1f), hff_f = fma(Pf2, c.p2f, Qf2 * c.q2f);
        const double hft_e = fma(Pf2, c.p3f, Qf2 * c.p4f), hft_f = fma(Pf2, c.p4f, -(Qf2 * c.p3f));
        const double htt_e = fma(Pt2, c.p1t, Qt2 * c.q1t), htt_f = fma(Pt2, c.p2t, Qt2 * c.q2t);
        const double htf_e = fma(Pt2, c.p3t, Qt2 * c.p4t), htf_f = fma(Pt2, c.p4t, -(Qt2 * c.p3t));
        if (fb < tb) {
            Jf[0] = hff_e; Jf[1] = hft_e; Jf[2] = hff_f; Jf[3] = hft_f;
            Jt[0] = htf_e; Jt[1] = htt_e; Jt[2] = htf_f; Jt[3] = htt_f;
        } else {
            Jf[0] = hft_e; Jf[1] = hff_e; Jf[2] = hft_f; Jf[3] = hff_f;
            Jt[0] = htt_e; Jt[1] = htf_e; Jt[2] = htt_f; Jt[3] = htf_f;
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
        if (l < N.nl) cart_branch_item<PS>(N, R, bl, l);
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

__device__ __forceinline__ void cart_bus_item(const DevNet &N, const CartReq &R, int bl, int i) {
    const int b = R.b0 + bl;
    const int nb = N.nb, ng = N.ng;
    const bool wantH = R.hval != nullptr;
    const double *scr = R.scratch + (size_t)bl * N.nslot * CNC;
    const int s0 = __ldg(N.slot_ptr + i), s1 = __ldg(N.slot_ptr + i + 1);
    const int k = __ldg(N.bus_k + i), nlow = __ldg(N.bus_nlow + i);
    double *Jb = R.jval ? R.jval + (size_t)b * R.nnzJc : nullptr;
    double *Hb = wantH ? R.hval + (size_t)b * N.nnzH : nullptr;
    double *JP = Jb ? Jb + __ldg(N.bus_jP + i) : nullptr;
    double *JQ = Jb ? Jb + __ldg(N.bus_jQ + i) : nullptr;
    double *HA = Hb ? Hb + __ldg(N.bus_hA + i) : nullptr;
    double *HM = Hb ? Hb + __ldg(N.bus_hM + i) : nullptr;

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
        ghb[i] = gP;
        ghb[nb + i] = gQ;
        ghb[2 * nb + 2 * N.nl + i] = V2;
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
        Jv[0] = twice(ei);
        Jv[1] = twice(fi);
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
                Hb[N.hpg + g] = gen_on(gm, g) ? sw * __ldg(N.c2g + g) : 0.0;
            }
        }
    }
    if (R.grad) {
        double *gb = R.grad + (size_t)b * N.n;
        gb[i] = 0.0;
        gb[nb + i] = 0.0;
        const double w = R.obj_weight ? __ldg(R.obj_weight + b) : 1.0;
        for (int q = g0; q < g1; q++) {
            const int g = __ldg(N.gen_ord + q);
            gb[2 * nb + g] = gen_on(gm, g) ? w * fma(__ldg(N.c2g + g), __ldg(xb + 2 * nb + g),
                                                     __ldg(N.c1g + g))
                                           : 0.0;
            gb[2 * nb + ng + g] = 0.0;
        }
    }
}

__global__ void __launch_bounds__(128) k_cart_bus(const DevNet N, const CartReq R, int nB) {
    const int per = (N.nb + 127) / 128;
    for (int it = blockIdx.x; it < nB * per; it += gridDim.x) {
        const int bl = it / per;
        const int i = (it - bl * per) * 128 + threadIdx.x;
        if (i < N.nb) cart_bus_item(N, R, bl, i);
    }
}

// Objective of each state (the polar model's: it depends on Pg only).
__global__ void __launch_bounds__(OBJ_LANES) k_cart_obj(const DevNet N, const EvalReq R, int b0) {
    __shared__ double part[OBJ_LANES];
    obj_block<true>(N, R, b0 + blockIdx.x, part);
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

}  // namespace
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
    const int chunk = B == 0 ? 0 : chunk_states(*dev, B);
    const int ring = chunk == 0 ? 0 : std::min(kRing, (B + chunk - 1) / chunk);
    *bytes = (size_t)ring * chunk * record_bytes(*dev);
    return EXAGO_OK;
}

exago_status exago_eval_cart(exago_net_t net, const exago_batch *bt, double *f, double *grad,
                             double *gh, double *jval, double *hval) {
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
    if (f) {
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
