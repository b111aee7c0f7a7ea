"""Mutation check of the oracle's pins.

Each mutant below is one plausible mistake in the oracle's own source (a
dropped factor, a flipped sign, a wrong index or factor, a transposed
operand).  The mutant is built by editing the source text of one oracle
function or method, compiled into a scratch namespace and patched in for the
duration of the check.  Every mutant must make at least one pin of
tests/test_oracle_*.py fail; the unmutated oracle must pass them all.  The
mistakes are planted in the oracle only, on the CPU.
"""
import importlib.util
import inspect
import os
import textwrap

import numpy as np
import pytest

import oracle
import oracle.dg2d as D
from synth import jittered_delaunay_mesh

HERE = os.path.dirname(os.path.abspath(__file__))


def _load(name):
    spec = importlib.util.spec_from_file_location("_pins_" + name, os.path.join(HERE, name + ".py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


RHS = _load("test_oracle_rhs")
ELEM = _load("test_oracle_element")
MESH = _load("test_oracle_mesh")
LSRK = _load("test_oracle_lsrk")
MEDIA = _load("test_oracle_media")
SRC = _load("test_oracle_source")
JIT4 = jittered_delaunay_mesh(4, seed=5)

MEDIA_PIN_UNIT = MEDIA.test_unit_permittivity_is_the_homogeneous_upwind_rhs
MEDIA_PIN_RIEMANN = MEDIA.test_interface_flux_is_the_riemann_solution

# pins, cheapest first; each is a call that raises when the pin fails
PINS = [
    ("lsrk order conditions", LSRK.test_order_conditions_up_to_four),
    ("lsrk stage times", LSRK.test_stage_times_consistent_with_butcher_rows),
    ("lsrk stability polynomial", LSRK.test_linear_stability_polynomial),
    ("Dr/Ds exact on polynomials", lambda: ELEM.test_dr_ds_differentiate_polynomials_exactly(3)),
    ("mass matrix exact", lambda: ELEM.test_mass_matrix_integrates_products_exactly(3)),
    ("LIFT face integrals", lambda: ELEM.test_lift_reproduces_face_integrals(3)),
    ("geometry", lambda: MESH.test_geometry_pins(3)),
    ("trace maps", lambda: MESH.test_trace_maps(2)),
    ("constant H steady", lambda: RHS.test_constant_magnetic_field_is_steady(JIT4)),
    ("volume exactness", lambda: RHS.test_volume_part_is_exact_for_polynomials(4, JIT4)),
    ("full rhs exactness", lambda: RHS.test_full_rhs_exact_for_continuous_polynomial_with_pec_zero(4)),
    ("1D Riemann flux", RHS.test_upwind_flux_matches_1d_riemann_solution),
    ("energy rate signs", lambda: RHS.test_energy_rate_signs(JIT4)),
    ("operator spectrum", lambda: RHS.test_brute_force_operator_spectrum(2)),
    ("permutation invariance", RHS.test_permutation_invariance),
    ("cavity mode", RHS.test_cavity_mode_config_one),
    ("media: unit eps", MEDIA_PIN_UNIT),
    ("media: interface Riemann", MEDIA_PIN_RIEMANN),
    ("media: dissipative weighted operator", lambda: MEDIA.test_weighted_operator_is_dissipative(2)),
    ("ricker closed forms", SRC.test_ricker_closed_forms),
    ("point source point values", lambda: SRC.test_point_source_reproduces_point_values(3)),
]


def _mutated(obj, old, new, count=1):
    """Compile `obj` (a function or method of oracle.dg2d) with `old`
    replaced by `new` in its source; returns the new function."""
    src = textwrap.dedent(inspect.getsource(obj))
    assert src.count(old) >= count, (obj.__name__, old)
    src = src.replace(old, new) if count == -1 else src.replace(old, new, count)
    ns = dict(D.__dict__)  # a copy: the module itself is left alone
    exec(compile(src, "<mutant of %s>" % obj.__qualname__, "exec"), ns)
    return ns[obj.__name__]


def _patch_function(mp, name, fn):
    mp.setattr(D, name, fn)
    if hasattr(oracle, name):
        mp.setattr(oracle, name, fn)


def _patch_method(mp, cls, name, fn):
    mp.setattr(cls, name, fn)


# (id, how to apply it); each entry plants one mistake
def _rhs(old, new, count=1):
    return lambda mp: _patch_function(mp, "maxwell_rhs", _mutated(D.maxwell_rhs, old, new, count))


def _disc(old, new):
    return lambda mp: _patch_method(mp, D.Discretization, "__init__",
                                    _mutated(D.Discretization.__init__, old, new))


def _ref(old, new):
    return lambda mp: _patch_method(mp, D.ReferenceElement, "__init__",
                                    _mutated(D.ReferenceElement.__init__, old, new))


def _media(old, new):
    return lambda mp: _patch_function(mp, "maxwell_rhs_media",
                                      _mutated(D.maxwell_rhs_media, old, new))


def _src(fn, old, new):
    return lambda mp: _patch_function(mp, fn, _mutated(getattr(D, fn), old, new))


def _lsrk_b_digit(mp):
    b = D.LSRK_B.copy()
    b[2] *= 1.0 + 1e-9  # one wrong digit in a coefficient
    mp.setattr(D, "LSRK_B", b)
    mp.setattr(oracle, "LSRK_B", b)


def _lsrk_published_c(mp):
    mp.setattr(D, "LSRK_C", D.LSRK_C_PUBLISHED.copy())
    mp.setattr(oracle, "LSRK_C", D.LSRK_C_PUBLISHED.copy())


MUTANTS = [
    ("flux factor 1/2 dropped", _rhs("@ R.LIFT.T / 2.0", "@ R.LIFT.T / 1.0", -1)),
    ("upwind H term sign", _rhs("alpha * (ndotdH * nx - dHx)", "alpha * (ndotdH * nx + dHx)")),
    ("upwind Ez term sign", _rhs("- alpha * dEz", "+ alpha * dEz")),
    ("PEC ghost: Ez+ = Ez-", _rhs("dEz[d.mapB] = 2.0 *", "dEz[d.mapB] = 0.0 *")),
    ("PEC ghost: H+ = -H-", _rhs("dHx[d.mapB] = 0.0", "dHx[d.mapB] = 2.0 * Hx.reshape(-1)[d.vmapB]")),
    ("dHy/dt uses d/dy", _rhs("rhsHy = ddx(Ez)", "rhsHy = ddy(Ez)")),
    ("curl H sign", _rhs("rhsEz = ddx(Hy) - ddy(Hx)", "rhsEz = ddx(Hy) + ddy(Hx)")),
    ("flux normals swapped", _rhs("fEz = ny * dHx - nx * dHy", "fEz = nx * dHx - ny * dHy")),
    ("Dr transposed", _rhs("d.rx * (u @ R.Dr.T)", "d.rx * (u @ R.Dr)")),
    ("ry replaced by rx", _rhs("d.ry * (u @ R.Dr.T)", "d.rx * (u @ R.Dr.T)")),
    ("Fscale dropped on Hx", _rhs("(d.Fscale * fHx) @", "(fHx) @")),
    ("jump sign (q+ - q-)", _rhs("dEz = Ez.reshape(-1)[vM] - Ez.reshape(-1)[vP]",
                                 "dEz = Ez.reshape(-1)[vP] - Ez.reshape(-1)[vM]")),
    ("Fscale without 1/J", _disc("self.Fscale = self.sJ / J[:, Fm.reshape(-1)]", "self.Fscale = self.sJ")),
    ("sx sign", _disc("self.sx = -yr / J", "self.sx = yr / J")),
    ("no neighbour coupling", _disc("self.vmapP = vmapP", "self.vmapP = self.vmapM.copy()")),
    ("Dr from V instead of V^T", _ref("self.Dr = np.linalg.solve(self.V.T, Vr.T).T",
                                      "self.Dr = np.linalg.solve(self.V, Vr.T).T")),
    ("LIFT with V V instead of V V^T", _ref("self.LIFT = self.V @ (self.V.T @ E)",
                                            "self.LIFT = self.V @ (self.V @ E)")),
    ("mass matrix from V^T V", _ref("self.M = np.linalg.inv(self.V @ self.V.T)",
                                    "self.M = np.linalg.inv(self.V.T @ self.V)")),
    ("LSRK b coefficient digit", _lsrk_b_digit),
    ("LSRK published c4", _lsrk_published_c),
    ("media: Z+ and Z- swapped", _media("fEz = (ZP * jHt - jEz) / (ZM + ZP)",
                                        "fEz = (ZM * jHt - jEz) / (ZM + ZP)")),
    ("media: Ez not divided by eps", _media(") / eps[:, None]", ") / 1.0")),
    ("source: no 1/J", _src("point_source_weights", "/ d.J[k, 0]", "/ 1.0")),
    ("source: Lagrange values via V", _src("point_source_weights",
                                           "np.linalg.solve(R.V.T, psi)", "np.linalg.solve(R.V, psi)")),
    ("source: wrong reference coordinate", _src("locate_point", "2.0 * l3[k] - 1.0",
                                                "2.0 * l1[k] - 1.0")),
    ("ricker: factor 2 dropped", _src("ricker", "(1.0 - 2.0 * a)", "(1.0 - a)")),
]


def _failing_pins(stop_at_first=True):
    failed = []
    for name, pin in PINS:
        try:
            pin()
        except Exception as ex:  # an assertion, or a crash the mistake causes
            failed.append((name, type(ex).__name__))
            if stop_at_first:
                break
    return failed


def test_unmutated_oracle_passes_every_pin():
    assert _failing_pins(stop_at_first=False) == []


@pytest.mark.parametrize("mutant", [m[0] for m in MUTANTS])
def test_every_mutant_fails_a_pin(mutant, monkeypatch):
    apply = dict(MUTANTS)[mutant]
    apply(monkeypatch)
    failed = _failing_pins()
    assert failed, "no pin caught the mutant: %s" % mutant
