"""Mutation check of the oracle's pins (CPU only).

Each mutant is a plausible transcription mistake planted in a copy of the C oracle (a flipped sign,
a dropped term or factor, a wrong or swapped index, a unit slip).  The copy is compiled into a
temporary library and the pins of test_oracle.py are run against it; every mutant must fail at
least one pin.  This shows that the pins constrain every part of the oracle's arithmetic.
"""
import os

import pytest

from oracle import acopf
import test_oracle as T
import test_oracle_cartesian as TK
import test_oracle_genmask as TG
import test_oracle_slack as TS
import test_oracle_coupling as TC
import test_oracle_shift as TP

SRC = os.path.join(os.path.dirname(acopf.__file__), "acopf_oracle.c")

MUTANTS = {
    "reactive_sign": ("double c = Gm * sn - Bm * cs;", "double c = Gm * sn + Bm * cs;"),
    "active_sign": ("double a = Gm * cs + Bm * sn;", "double a = Gm * cs - Bm * sn;"),
    "dP_dVu_factor": ("dP[2] = 2.0 * Gss * Vu + Vv * a;", "dP[2] = Gss * Vu + Vv * a;"),
    "dQ_dVv_index": ("dQ[3] = Vu * c;", "dQ[3] = Vv * c;"),
    "HP_mixed_index": ("HP[i * 4 + 3] = HP[3 * 4 + i] = Vu * (-c) * e[i];",
                       "HP[i * 4 + 3] = HP[3 * 4 + i] = Vv * (-c) * e[i];"),
    "HQ_angle_term": ("HQ[i * 4 + j] = VV * (-c) * e[i] * e[j];",
                      "HQ[i * 4 + j] = VV * (-a) * e[i] * e[j];"),
    "HQ_self_sign": ("HQ[2 * 4 + 2] = -2.0 * Bss;", "HQ[2 * 4 + 2] = 2.0 * Bss;"),
    "hess_dropped_outer": ("+ dQ[a] * dQ[bb] + Q * HQ[a * 4 + bb]);", "+ Q * HQ[a * 4 + bb]);"),
    "hess_mu_factor": ("+ mu * 2.0 * (dP[a]", "+ mu * (dP[a]"),
    "to_side_swapped": ("gidx[1][0] = tb; gidx[1][1] = fb;", "gidx[1][0] = fb; gidx[1][1] = tb;"),
    "charging_not_halved": ("Y[1] = (bs + 0.5 * b) / (tau * tau);", "Y[1] = (bs + b) / (tau * tau);"),
    "tap_square_mutual": ("Y[2] = -(gs * cp - bs * sp) / tau;", "Y[2] = -(gs * cp - bs * sp) / (tau * tau);"),
    "shift_ft_conjugate": ("Y[2] = -(gs * cp - bs * sp) / tau;",
                           "Y[2] = -(gs * cp + bs * sp) / tau;"),
    "shift_tf_sign": ("Y[5] = -(bs * cp - gs * sp) / tau;", "Y[5] = -(bs * cp + gs * sp) / tau;"),
    "shift_ends_equal": ("Y[4] = -(gs * cp + bs * sp) / tau;", "Y[4] = -(gs * cp - bs * sp) / tau;"),
    "shift_dropped_in_Bft": ("Y[3] = -(gs * sp + bs * cp) / tau;", "Y[3] = -(bs * cp) / tau;"),
    "shift_ignored": ("return net->shift ? net->shift[l] : 0.0;", "return 0.0;"),
    "shift_on_tap_magnitude": ("Y[0] = gs / (tau * tau);", "Y[0] = gs * cp / (tau * tau);"),
    "tap_on_wrong_end": ("Y[6] = gs;", "Y[6] = gs / (tau * tau);"),
    "h_jac_factor": ("2.0 * P * dP[a] + 2.0 * Q * dQ[a]", "P * dP[a] + Q * dQ[a]"),
    "cost_units": ("net->c1[k] * MW + net->c0[k]", "net->c1[k] * Pg[k] + net->c0[k]"),
    "grad_units": ("+ net->c1[k] * base);", "+ net->c1[k]);"),
    "hess_sigma": ("sigma * w * 2.0 * net->c2[k]", "w * 2.0 * net->c2[k]"),
    "shunt_hess_sign": ("- lamQ[i] * 2.0 * net->Bs[i])) return -2;", "+ lamQ[i] * 2.0 * net->Bs[i])) return -2;"),
    "shunt_jac_dropped": ("if (push(J, i, nb + i, 2.0 * net->Gs[i] * Vm[i])) return -2;",
                          "if (push(J, i, nb + i, 0.0)) return -2;"),
    "load_scale_dropped": ("Vm[i] * Vm[i] + net->Pd[i] * sc;", "Vm[i] * Vm[i] + net->Pd[i];"),
    "mask_ignored": ("P *= m;", "P *= 1.0;"),
    "gen_q_on_p_row": ("gQ[gb] -= Qg[k];", "gP[gb] -= Qg[k];"),
    "cart_db_sign": ("const double db[4] = {-fv, ev, fu, -eu};", "const double db[4] = {fv, ev, fu, -eu};"),
    "cart_Hb_sign": ("Hb[16] = {0, 0, 0, -1,", "Hb[16] = {0, 0, 0, 1,"),
    "cart_Ha_index": ("Ha[16] = {0, 0, 1, 0,  0, 0, 0, 1,", "Ha[16] = {0, 1, 0, 0,  1, 0, 0, 1,"),
    "cart_Q_sign": ("*Q = -Bss * s + Gm * b - Bm * a;", "*Q = -Bss * s + Gm * b + Bm * a;"),
    "cart_ds_factor": ("const double ds[4] = {2.0 * eu, 2.0 * fu, 0.0, 0.0};",
                       "const double ds[4] = {eu, fu, 0.0, 0.0};"),
    "cart_voltage_row": ("if (push(J, vrow, nb + i, 2.0 * F[i])) return -2;",
                         "if (push(J, vrow, nb + i, F[i])) return -2;"),
    "cart_muV_hess": ("+ muV[i] * 2.0;", "+ muV[i];"),
    "cart_shunt_f": ("if (push(J, nb + i, nb + i, -2.0 * net->Bs[i] * F[i])) return -2;",
                     "if (push(J, nb + i, nb + i, -2.0 * net->Bs[i] * E[i])) return -2;"),
    "cart_to_side": ("gidx[1][2] = fb; gidx[1][3] = nb + fb;", "gidx[1][2] = nb + fb; gidx[1][3] = fb;"),
    "gen_mask_ignored": ("int on = gmask == NULL || gmask[k] != 0;", "int on = 1;"),
    "gen_mask_jac_kept": ("if (push(J, gb, 2 * nb + k, on ? -1.0 : 0.0)) return -2;",
                          "if (push(J, gb, 2 * nb + k, -1.0)) return -2;"),
    "gen_mask_hess_kept": ("double hk = on ? sigma", "double hk = 1 ? sigma"),
    "slack_sign_dropped": ("gh[row[k] * nb + bus[k]] += sign[k] * z[k];", "gh[row[k] * nb + bus[k]] += z[k];"),
    "slack_row_dropped": ("gh[row[k] * nb + bus[k]] += sign[k]", "gh[bus[k]] += sign[k]"),
    "slack_weight_dropped": ("if (f) *f += w * cost[k] * z[k];", "if (f) *f += cost[k] * z[k];"),
    "coupling_sign": ("x[(int64_t)b * n + 2 * nb + k] - x[(int64_t)p * n + 2 * nb + k]",
                      "x[(int64_t)b * n + 2 * nb + k] + x[(int64_t)p * n + 2 * nb + k]"),
    "coupling_parent_stride": ("- x[(int64_t)p * n + 2 * nb + k]", "- x[(int64_t)p * ng + 2 * nb + k]"),
    "coupling_root_row": ("p < 0 ? 0.0 :", "p < 0 ? x[(int64_t)b * n + 2 * nb + k] :"),
    "coupling_jtv_parent_sign": ("out[(int64_t)p * n + 2 * nb + k] -=", "out[(int64_t)p * n + 2 * nb + k] +="),
    "coupling_jtv_offset": ("out[(int64_t)b * n + 2 * nb + k] +=", "out[(int64_t)b * n + nb + k] +="),
}


class Bound:
    """The oracle module's API bound to one compiled library."""

    def __init__(self, lib):
        self.lib = lib
        self.OracleNet = acopf.OracleNet
        self.csr_to_dense = acopf.csr_to_dense

    def evaluate(self, *a, **k):
        return acopf.evaluate(*a, lib=self.lib, **k)

    def slack(self, *a, **k):
        return acopf.slack(*a, lib=self.lib, **k)

    def coupling(self, *a, **k):
        return acopf.coupling(*a, lib=self.lib, **k)

    def coupling_jtv(self, *a, **k):
        return acopf.coupling_jtv(*a, lib=self.lib, **k)


PINS = [
    ("power_angle", lambda om: T.test_power_angle_equations_lossless_line(om)),
    ("transformer", lambda om: T.test_transformer_scales_from_voltage(om)),
    ("flat_start", lambda om: T.test_flat_start(om)),
    ("objective", lambda om: T.test_objective_hand_numbers(om)),
    ("nodal_3", lambda om: T.test_matches_complex_nodal_form(om, 21, 3, 3, 1, 0.0)),
    ("nodal_30", lambda om: T.test_matches_complex_nodal_form(om, 22, 30, 41, 6, 0.0)),
    ("loss", lambda om: T.test_loss_invariant(om, 0.0)),
    ("loss_shift", lambda om: T.test_loss_invariant(om, 0.3)),
    ("fd", lambda om: T.test_finite_differences(om, 41)),
    ("fd_sigma0", lambda om: T.test_finite_differences_sigma_zero_and_transformers(om)),
    ("mask", lambda om: T.test_mask_equals_branch_removed(om)),
    ("symmetries", lambda om: T.test_homogeneity_and_angle_invariance(om)),
    ("cart_nodal", lambda om: TK.test_matches_complex_nodal_form(om)),
    ("cart_polar", lambda om: TK.test_change_of_variables_to_polar(om, 53)),
    ("cart_fd", lambda om: TK.test_finite_differences(om)),
    ("cart_homogeneity", lambda om: TK.test_homogeneity_and_rotation(om)),
    ("gen_out_polar", lambda om: TG.test_generator_out_equals_generator_removed(om, False)),
    ("gen_out_hand", lambda om: TG.test_two_bus_generator_outage_by_hand(om)),
    ("slack_hand", lambda om: TS.test_hand_values(om)),
    ("slack_load_loss", lambda om: TS.test_load_loss_equals_lower_load(om)),
    ("shift_closed_form", lambda om: TP.test_lossless_phase_shifter_closed_form(om)),
    ("shift_rotation", lambda om: TP.test_shift_equals_rotated_from_angle(om, 0.02, 0.12, 0.05, 1.0, 0.35)),
    ("shift_nodal", lambda om: T.test_matches_complex_nodal_form(om, 24, 60, 80, 12, 0.25)),
    ("shift_cart", lambda om: TP.test_cartesian_change_of_variables_with_shifters(om)),
    ("coupling_hand", lambda om: TC.test_hand_rows(om)),
    ("coupling_hand_transpose", lambda om: TC.test_hand_transpose(om)),
    ("coupling_telescopes", lambda om: TC.test_chain_telescopes(om)),
    ("coupling_transpose", lambda om: TC.test_transpose_identity(om, 9, 40, 5)),
]


def test_unmutated_copy_passes_all_pins(tmp_path):
    lib = acopf.bind_library(acopf.compile_source(SRC, str(tmp_path / "good.so")))
    for name, pin in PINS:
        pin(Bound(lib))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    lib = acopf.bind_library(acopf.compile_source(str(path), str(tmp_path / f"{name}.so")))
    caught = []
    for pname, pin in PINS:
        try:
            pin(Bound(lib))
        except (AssertionError, ValueError):
            caught.append(pname)
    assert caught, f"mutant {name} passed every pin"
