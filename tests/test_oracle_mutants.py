"""The oracle's pins must catch plausible mistakes. Each case plants one mistake
in a temporary copy of the oracle's C source (never in the committed file),
builds it with gcc, swaps it in, and checks that a pin now fails."""
import os
import subprocess

import pytest

import tests.test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "qv_oracle.c")

MUTANTS = [
    ("eq5_transposed_operand",
     "        psi[i] = U[0] * a + U[1] * b;\n        psi[j] = U[2] * a + U[3] * b;\n    }\n}\n\n/* Controlled",
     "        psi[i] = U[0] * a + U[2] * b;\n        psi[j] = U[1] * a + U[3] * b;\n    }\n}\n\n/* Controlled",
     lambda O: pins.test_apply_1q_equals_kronecker(O, 3)),
    ("eq5_pairs_bit_set",
     "        if (i & bit) continue;\n        const uint64_t j = i ^ bit;",
     "        if (!(i & bit)) continue;\n        const uint64_t j = i ^ bit;",
     lambda O: pins.test_apply_1q_equals_kronecker(O, 3)),
    ("u3_sign",
     "U[1] = -cexp(I * la) * sin(th / 2);",
     "U[1] = cexp(I * la) * sin(th / 2);",
     lambda O: pins.test_gate_matrix_textbook_values(O)),
    ("u3_phase_swapped",
     "U[2] = cexp(I * ph) * sin(th / 2);",
     "U[2] = cexp(I * la) * sin(th / 2);",
     lambda O: pins.test_gate_matrix_textbook_values(O)),
    ("rz_sign",
     "U[0] = cexp(-I * th / 2); U[1] = 0; U[2] = 0; U[3] = cexp(I * th / 2);",
     "U[0] = cexp(I * th / 2); U[1] = 0; U[2] = 0; U[3] = cexp(-I * th / 2);",
     lambda O: pins.test_gate_matrix_textbook_values(O)),
    ("ry_half_angle_dropped",
     "U[0] = cos(th / 2); U[1] = -sin(th / 2);\n        U[2] = sin(th / 2); U[3] = cos(th / 2);",
     "U[0] = cos(th); U[1] = -sin(th);\n        U[2] = sin(th); U[3] = cos(th);",
     lambda O: pins.test_gate_matrix_textbook_values(O)),
    ("control_polarity",
     "        if (!(i & cbit)) continue;",
     "        if (i & cbit) continue;",
     lambda O: pins.test_controlled_equals_dense(O, 3)),
    ("swap_wrong_partner",
     "            const uint64_t j = (i ^ ba) | bb;",
     "            const uint64_t j = i ^ bb;",
     lambda O: pins.test_swap_and_permute_equal_axis_transpose(O)),
    ("expect_z_bit_reversed",
     "            s += ((i >> q) & 1) ? -p : p;",
     "            s += ((i >> (n - 1 - q)) & 1) ? -p : p;",
     lambda O: pins.test_expect_z_product_state_closed_form(O)),
    ("pauli_y_phase_dropped",
     "    for (int y = 0; y < ny; ++y) iy *= I;\n    cplx s = 0;",
     "    for (int y = 0; y < ny; ++y) iy *= 1;\n    cplx s = 0;",
     lambda O: pins.test_expect_pauli_equals_dense(O)),
    ("pauli_conj_dropped",
     "        s += conj(psi[i ^ xmask]) * pi;",
     "        s += psi[i ^ xmask] * pi;",
     lambda O: pins.test_expect_pauli_equals_dense(O)),
    ("norm_drops_imag",
     "    for (uint64_t i = 0; i < dim; ++i) s += creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);",
     "    for (uint64_t i = 0; i < dim; ++i) s += creal(psi[i]) * creal(psi[i]);",
     lambda O: pins.test_norm_preserved_and_inverse_returns_input(O)),
]


@pytest.mark.parametrize("name,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_planted_mistake(tmp_path, monkeypatch, orc, name, old, new, pin):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor not found exactly once: " + name
    mutant_c = tmp_path / (name + ".c")
    mutant_c.write_text(src.replace(old, new))
    so = tmp_path / (name + ".so")
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", "-o", str(so), str(mutant_c), "-lm"])
    monkeypatch.setattr(orc, "_lib", orc.load(str(so)))
    with pytest.raises(AssertionError):
        pin(orc)
