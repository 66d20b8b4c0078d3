"""The SBML front end (the paper's Section 2: models are read from SBML files): exact
round trips of every workload network, a hand-written SBML Level 2 file of the
decaying-dimerizing set that the paper's Section 3 simulates (reversible difference law,
local parameters, e-notation, powers, a compartment factor), catalysts given as
modifiers, boundary species folded into the rate constant, and clear errors for what is
not a mass-action network."""
import os

import numpy as np
import pytest

from paper_1608_07058_gb300 import sbml, workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "decaying_dimerizing_l2.xml")


@pytest.mark.parametrize("crn,x0", [
    (W.immigration_death(), [0]), (W.dimerisation(), [400, 798, 0]),
    (W.gene_expression(), [0, 0, 0]), W.random_crn(seed=3), (W.isomerisation(), [7, 3])])
def test_round_trip(crn, x0):
    m = sbml.read_sbml(sbml.write_sbml(crn, x0))
    assert np.array_equal(m.crn.orders, crn.orders)
    assert np.array_equal(m.crn.stoich, crn.stoich)
    assert np.array_equal(m.crn.rates, crn.rates)
    assert np.array_equal(m.x0, np.asarray(x0, np.int64))


def test_golden_decaying_dimerizing_file():
    m = sbml.load_sbml(GOLDEN)
    ref = W.dimerisation()
    assert m.crn.species == ("S1", "S2", "S3")
    assert m.reaction_ids == ("decay", "dimerisation", "dimerisation_reverse", "conversion")
    assert np.array_equal(m.crn.orders, ref.orders)
    assert np.array_equal(m.crn.stoich, ref.stoich)
    assert np.array_equal(m.crn.rates, ref.rates)
    assert np.array_equal(m.x0, [400, 798, 0])


def test_golden_file_simulates_like_the_workload(oracle):
    m = sbml.load_sbml(GOLDEN)
    a = oracle.simulate(m.crn, 50, m.x0, [0.2], seed=8)
    b = oracle.simulate(W.dimerisation(), 50, [400, 798, 0], [0.2], seed=8)
    assert np.array_equal(a["X"], b["X"]) and np.array_equal(a["r"], b["r"])


def _doc(species, reactions, params=""):
    return f"""<sbml xmlns="http://www.sbml.org/sbml/level3/version1/core" level="3" version="1">
<model id="t"><listOfCompartments><compartment id="c" size="2"/></listOfCompartments>
<listOfSpecies>{species}</listOfSpecies>
<listOfParameters>{params}</listOfParameters>
<listOfReactions>{reactions}</listOfReactions></model></sbml>"""


MATH = '<math xmlns="http://www.w3.org/1998/Math/MathML">{}</math>'
SP = '<species id="{}" compartment="c" initialAmount="{}" {}/>'


def _rx(rid, reac, prod, law, mods="", extra=""):
    r = "".join(f'<speciesReference species="{s}" stoichiometry="{m}"/>' for s, m in reac)
    p = "".join(f'<speciesReference species="{s}" stoichiometry="{m}"/>' for s, m in prod)
    md = "".join(f'<modifierSpeciesReference species="{s}"/>' for s in mods)
    return (f'<reaction id="{rid}" reversible="false">'
            + (f"<listOfReactants>{r}</listOfReactants>" if r else "")
            + (f"<listOfProducts>{p}</listOfProducts>" if p else "")
            + (f"<listOfModifiers>{md}</listOfModifiers>" if md else "")
            + f"<kineticLaw>{MATH.format(law)}{extra}</kineticLaw></reaction>")


def test_modifier_is_a_catalyst():
    sp = SP.format("G", 1, "") + SP.format("M", 0, "")
    rx = _rx("tx", [], [("M", 1)], "<apply><times/><ci>k</ci><ci>G</ci></apply>", mods=["G"])
    m = sbml.read_sbml(_doc(sp, rx, '<parameter id="k" value="10"/>'))
    assert m.crn.orders.tolist() == [[1, 0]] and m.crn.stoich.tolist() == [[0, 1]]
    assert m.crn.rates.tolist() == [10.0]


def test_boundary_species_folds_into_rate_and_compartment_factor():
    sp = SP.format("B", 5, 'boundaryCondition="true"') + SP.format("A", 9, "") + SP.format("C", 0, "")
    law = "<apply><times/><ci>c</ci><ci>k</ci><ci>A</ci><apply><power/><ci>B</ci><cn>2</cn></apply></apply>"
    rx = _rx("r", [("A", 1), ("B", 2)], [("C", 1)], law)
    m = sbml.read_sbml(_doc(sp, rx, '<parameter id="k" value="0.5"/>'))
    assert m.crn.species == ("A", "C")
    assert m.crn.orders.tolist() == [[1, 0]] and m.crn.stoich.tolist() == [[-1, 1]]
    assert m.crn.rates[0] == pytest.approx(2 * 0.5 * 10)   # compartment 2, C(5, 2) = 10
    assert m.x0.tolist() == [9, 0]


def test_local_parameter_and_division_by_constant():
    sp = SP.format("A", 3, "")
    law = "<apply><divide/><apply><times/><ci>k</ci><ci>A</ci></apply><cn>4</cn></apply>"
    extra = '<listOfLocalParameters><localParameter id="k" value="8"/></listOfLocalParameters>'
    m = sbml.read_sbml(_doc(sp, _rx("d", [("A", 1)], [], law, extra=extra)))
    assert m.crn.rates.tolist() == [2.0]


@pytest.mark.parametrize("law,reac,msg", [
    ("<apply><divide/><apply><times/><ci>k</ci><ci>A</ci></apply>"
     "<apply><plus/><ci>k</ci><ci>A</ci></apply></apply>", [("A", 1)], "not supported"),
    ("<apply><times/><ci>k</ci><ci>A</ci><ci>A</ci></apply>", [("A", 1)], "not mass action"),
    ("<apply><times/><ci>k</ci><ci>Z</ci></apply>", [("A", 1)], "unknown identifier"),
    ("<apply><times/><ci>k</ci><apply><power/><ci>A</ci><cn>4</cn></apply></apply>",
     [("A", 4)], "order above 3"),
    ("<apply><exp/><ci>A</ci></apply>", [("A", 1)], "not supported"),
])
def test_rejects_non_mass_action(law, reac, msg):
    sp = SP.format("A", 3, "") + SP.format("C", 0, "")
    with pytest.raises(sbml.SBMLError, match=msg):
        sbml.read_sbml(_doc(sp, _rx("r", reac, [("C", 1)], law), '<parameter id="k" value="1"/>'))


def test_rejects_fractional_stoichiometry_events_and_garbage():
    sp = SP.format("A", 3, "")
    bad = _rx("r", [("A", 1.5)], [], "<ci>k</ci>")
    with pytest.raises(sbml.SBMLError, match="stoichiometry"):
        sbml.read_sbml(_doc(sp, bad, '<parameter id="k" value="1"/>'))
    ev = _doc(sp, _rx("r", [("A", 1)], [], "<apply><times/><ci>k</ci><ci>A</ci></apply>"),
              '<parameter id="k" value="1"/>').replace(
        "</listOfReactions>", "</listOfReactions><listOfEvents><event id='e'/></listOfEvents>")
    with pytest.raises(sbml.SBMLError, match="listOfEvents"):
        sbml.read_sbml(ev)
    with pytest.raises(sbml.SBMLError, match="not XML"):
        sbml.read_sbml("<sbml")


def test_parsed_model_goes_to_the_library():
    from paper_1608_07058_gb300 import build, matleap
    build.build()
    m = sbml.load_sbml(GOLDEN)
    model = matleap.model_from_crn(m.crn)
    assert matleap.ml_model_num_pairs(model) == 1
    assert model.N == 3 and model.M == 4


def test_round_trip_random_networks():
    """Any mass-action network (orders up to 3, products up to 3 per species, rates over
    many decades, zero-order sources) survives write_sbml -> read_sbml exactly."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=60, deadline=None)
    @hyp.given(st.data())
    def check(data):
        N = data.draw(st.integers(1, 6))
        M = data.draw(st.integers(1, 8))
        reactions = []
        for _ in range(M):
            re, pr, total = {}, {}, 0
            for s in range(N):
                m = data.draw(st.integers(0, 3 - total))
                if m:
                    re[s] = m
                    total += m
                q = data.draw(st.integers(0, 3))
                if q:
                    pr[s] = q
            k = data.draw(st.floats(1e-12, 1e12, allow_nan=False, allow_infinity=False))
            reactions.append((re, pr, k))
        crn = W._crn("random", N, reactions, tuple(f"X{s}" for s in range(N)))
        x0 = data.draw(st.lists(st.integers(0, 10**12), min_size=N, max_size=N))
        m = sbml.read_sbml(sbml.write_sbml(crn, x0))
        assert np.array_equal(m.crn.orders, crn.orders)
        assert np.array_equal(m.crn.stoich, crn.stoich)
        assert np.array_equal(m.crn.rates, crn.rates)
        assert np.array_equal(m.x0, np.asarray(x0, np.int64))

    check()
