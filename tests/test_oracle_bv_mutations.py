"""Mutation check of the Butler-Volmer oracle's pins (no GPU).

Each case plants one plausible mistake in a copy of oracle/bv.py (a sign, an exponent, a
stoichiometric number, a boundary term, the electroneutrality closure) and runs the pin
of tests/test_oracle_bv.py named beside it against the copy: the pin must fail. The
unmodified copy passes every named pin.
"""
import os
import sys
import types

import pytest

import tests.test_oracle_bv as pins

SOURCE_PATH = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                           "oracle", "bv.py")

MUTATIONS = [
    ("migration_sign",
     [("g = z * D * soc.FARADAY / (soc.R_GAS * p.T * p.h * p.h)",
       "g = -z * D * soc.FARADAY / (soc.R_GAS * p.T * p.h * p.h)")],
     "test_fixed_point_balances_every_species_and_the_counter_ion", {}),
    ("membrane_flux_sign",
     [("vals = np.concatenate([vals, -2.0 * g * phi[m]])",
       "vals = np.concatenate([vals, 2.0 * g * phi[m]])")],
     "test_fixed_point_balances_every_species_and_the_counter_ion", {}),
    ("conductivity_with_z_not_z_squared",
     [("kcell = pre * sum(Z[k] ** 2 * Dk[k] * C[k] for k in (\"O\", \"R\", \"H\", \"X\"))",
       "kcell = pre * sum(abs(Z[k]) * Dk[k] * C[k] for k in (\"O\", \"R\", \"H\", \"X\"))")],
     "test_fixed_point_balances_every_species_and_the_counter_ion", {}),
    ("one_proton_per_reaction",
     [("N_STOICH = {\"O\": -1.0, \"R\": 1.0, \"H\": -2.0}",
       "N_STOICH = {\"O\": -1.0, \"R\": 1.0, \"H\": -1.0}")],
     "test_fixed_point_balances_every_species_and_the_counter_ion", {}),
    ("ionic_diffusion_term_sign",
     [("acc = acc - soc.FARADAY * Z[k] * Dk[k] * (L @ C[k] + b)",
       "acc = acc + soc.FARADAY * Z[k] * Dk[k] * (L @ C[k] + b)")],
     "test_fixed_point_balances_every_species_and_the_counter_ion", {}),
    ("counter_ion_one_charge_per_quinone",
     [("return C[\"H\"] - 2.0 * (C[\"O\"] + C[\"R\"])", "return C[\"H\"] - (C[\"O\"] + C[\"R\"])")],
     "test_fixed_point_balances_every_species_and_the_counter_ion", {}),
    ("quinone_crosses_the_membrane",
     [("AO = LO + migration(p, Z[\"O\"], Dk[\"O\"], phi, False)",
       "AO = LO + migration(p, Z[\"O\"], Dk[\"O\"], phi, True)")],
     "test_fixed_point_balances_every_species_and_the_counter_ion", {}),
    ("transfer_coefficients_swapped",
     [("return kap * np.exp(p.alpha * vc), kap * np.exp((p.alpha - 1.0) * vc)",
       "return kap * np.exp((1.0 - p.alpha) * vc), kap * np.exp(-p.alpha * vc)")],
     "test_source_is_the_butler_volmer_rate", {"alpha": 0.3}),
    ("electrolyte_potential_sign",
     [("vc = kin.Vt + p.n_e * phi / kin.V_T", "vc = kin.Vt - p.n_e * phi / kin.V_T")],
     "test_source_is_the_butler_volmer_rate", {"alpha": 0.5}),
    ("inlet_quinones_swapped",
     [("cO, cR = (1.0 - p.s_in) * p.c0, p.s_in * p.c0", "cO, cR = p.s_in * p.c0, (1.0 - p.s_in) * p.c0")],
     "test_zero_potential_step_is_the_sbv_model", {}),
    ("reduced_species_gains_from_the_back_reaction",
     [("[sp.diags(kf), AR - sp.diags(kb)]", "[sp.diags(kf), AR + sp.diags(kb)]")],
     "test_zero_potential_step_is_the_sbv_model", {}),
    ("membrane_conductance_all_ions",
     [("km = pre * Dk[\"H\"] * C[\"H\"][m] / (p.h * p.h)", "km = kcell[m] / (p.h * p.h)")],
     "test_fixed_point_balances_every_species_and_the_counter_ion", {}),
]


def _load(edits, tag):
    src = open(SOURCE_PATH).read()
    for old, new in edits:
        assert src.count(old) == 1, "edit target not found once: %r" % old
        src = src.replace(old, new)
    src = src.replace("from . import soc", "from oracle import soc")
    name = "oracle_bv_mutant_%s" % tag
    mod = types.ModuleType(name)
    mod.__file__ = SOURCE_PATH
    sys.modules[name] = mod
    exec(compile(src, SOURCE_PATH, "exec"), mod.__dict__)
    return mod


def _run_pin(monkeypatch, mod, pin, kwargs):
    monkeypatch.setattr(pins, "bv", mod)
    for f in (pins._solved,):
        f.cache_clear()
    try:
        getattr(pins, pin)(**kwargs)
        return None
    except AssertionError:
        return "assertion"
    except RuntimeError as e:
        assert "did not converge" in str(e), "planted edit broke the copy: %r" % e
        return "non-convergence"
    finally:
        pins._solved.cache_clear()


def test_unmodified_copy_passes_every_named_pin(monkeypatch):
    mod = _load([], "unmodified")
    try:
        seen = set()
        for _, _, pin, kwargs in MUTATIONS:
            key = (pin, tuple(sorted(kwargs.items())))
            if key not in seen:
                seen.add(key)
                assert _run_pin(monkeypatch, mod, pin, kwargs) is None, key
    finally:
        del sys.modules[mod.__name__]


@pytest.mark.parametrize("name,edits,pin,kwargs", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_its_pin(monkeypatch, name, edits, pin, kwargs):
    mod = _load(edits, name)
    try:
        import warnings
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")
            why = _run_pin(monkeypatch, mod, pin, kwargs)
    finally:
        del sys.modules[mod.__name__]
    assert why is not None, "%s: %s still passes" % (name, pin)
