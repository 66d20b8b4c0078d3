"""Model front end: mass-action networks from SBML (the paper, Section 2: models are given
as SBML files) and back.

The reader covers the part of SBML Level 2/3 core that describes a mass-action network:

- species with an initial amount (or concentration, taken as a count) and the
  boundaryCondition / constant flags;
- global parameters, compartments (a compartment id in a law counts as its size) and a
  reaction's local parameters;
- reactions with reactant / product species references and integer stoichiometries, and
  modifiers;
- kinetic laws whose MathML is a product of numbers, parameters, compartments and species
  (species may appear as powers), or, for reversible reactions, the difference of two such
  products.

Readings (the paper does not describe its SBML import):

- The law's coefficient is the stochastic rate constant theta_j.  Its species factors must
  match the reactant multiplicities, but they are not evaluated as written: the
  propensity is always theta_j prod_s C(x_s, m_js), the convention of the simulator.
- A reversible law "k_f * reactants - k_r * products" becomes two reactions, the forward
  one and its reverse, which the simulator then recognises as a reversible pair.
- A modifier that appears in the law (with power e) is a catalyst: reactant and product
  with multiplicity e.
- A boundary or constant species never changes.  Its count C(x_b, m) is folded into
  theta_j, and it is left out of the state.

Anything else raises SBMLError with the offending element named: events, rules, function
definitions, non-integer stoichiometry, and laws that are not mass action.  Python, off
the simulation path: the result is a workloads.CRN plus the initial state, which
ml_model_create takes as plain arrays.
"""
from __future__ import annotations

import math
import xml.etree.ElementTree as ET
from dataclasses import dataclass
from typing import Dict, List, Tuple

import numpy as np

from .workloads import CRN


class SBMLError(ValueError):
    pass


@dataclass
class SBMLModel:
    crn: CRN
    x0: np.ndarray          # initial counts, int64, in crn.species order
    reaction_ids: tuple     # one id per CRN reaction ("<id>" or "<id>_reverse")


def _local(tag: str) -> str:
    return tag.rsplit("}", 1)[-1]


def _children(el, name):
    return [c for c in el if _local(c.tag) == name]


def _child(el, name):
    for c in el:
        if _local(c.tag) == name:
            return c
    return None


def _items(el, list_name, item_name):
    """The <item_name> children of el's <list_name> child (none if the list is absent)."""
    lst = _child(el, list_name)
    return [] if lst is None else _children(lst, item_name)


def _int_stoich(ref, where) -> int:
    v = ref.get("stoichiometry")
    if v is None:
        math_el = _child(ref, "stoichiometryMath")
        if math_el is not None:
            raise SBMLError(f"{where}: stoichiometryMath is not supported")
        return 1
    f = float(v)
    if f != int(f) or f < 0:
        raise SBMLError(f"{where}: stoichiometry {v} is not a non-negative integer")
    return int(f)


# A mass-action term: coefficient times prod species^power.
Term = Tuple[float, Dict[str, int]]


def _eval(node, symbols: Dict[str, float], species: set, where: str) -> List[Term]:
    """MathML to a sum of terms (at most two, for a reversible law)."""
    tag = _local(node.tag)
    if tag == "math":
        kids = list(node)
        if len(kids) != 1:
            raise SBMLError(f"{where}: the law must be one expression")
        return _eval(kids[0], symbols, species, where)
    if tag == "cn":
        txt = (node.text or "").strip()
        kind = node.get("type", "real")
        if kind == "e-notation":
            parts = [t.strip() for t in node.itertext() if t.strip()]
            val = float(parts[0]) * 10.0 ** float(parts[1])
        elif kind == "rational":
            parts = [t.strip() for t in node.itertext() if t.strip()]
            val = float(parts[0]) / float(parts[1])
        else:
            val = float(txt)
        return [(val, {})]
    if tag == "ci":
        name = (node.text or "").strip()
        if name in species:
            return [(1.0, {name: 1})]
        if name in symbols:
            return [(symbols[name], {})]
        raise SBMLError(f"{where}: unknown identifier '{name}'")
    if tag != "apply":
        raise SBMLError(f"{where}: MathML element <{tag}> is not supported")
    kids = list(node)
    op = _local(kids[0].tag)
    args = [_eval(k, symbols, species, where) for k in kids[1:]]
    if op == "times":
        out: List[Term] = [(1.0, {})]
        for a in args:
            if len(a) != 1 or len(out) != 1:
                raise SBMLError(f"{where}: a product of sums is not mass action")
            c, p = out[0]
            c2, p2 = a[0]
            q = dict(p)
            for s, e in p2.items():
                q[s] = q.get(s, 0) + e
            out = [(c * c2, q)]
        return out
    if op == "power":
        if len(args) != 2 or len(args[0]) != 1 or len(args[1]) != 1 or args[1][0][1]:
            raise SBMLError(f"{where}: power needs a single base and a numeric exponent")
        (c, p), (e, _) = args[0][0], args[1][0]
        if e != int(e) or e < 0:
            raise SBMLError(f"{where}: exponent {e} is not a non-negative integer")
        e = int(e)
        return [(c ** e, {s: k * e for s, k in p.items()})]
    if op == "divide":
        if len(args) != 2 or len(args[1]) != 1 or args[1][0][1] or len(args[0]) != 1:
            raise SBMLError(f"{where}: only division by a constant is mass action")
        (c, p), (d, _) = args[0][0], args[1][0]
        return [(c / d, p)]
    if op == "minus":
        if len(args) == 2 and len(args[0]) == 1 and len(args[1]) == 1:
            return [args[0][0], (-args[1][0][0], args[1][0][1])]
        raise SBMLError(f"{where}: only 'forward - reverse' differences are supported")
    raise SBMLError(f"{where}: MathML operator <{op}> is not supported")


def read_sbml(text: str) -> SBMLModel:
    """Parse an SBML document (a string) into a CRN and its initial state."""
    try:
        root = ET.fromstring(text)
    except ET.ParseError as e:
        raise SBMLError(f"not XML: {e}") from None
    if _local(root.tag) != "sbml":
        raise SBMLError("root element is not <sbml>")
    model = _child(root, "model")
    if model is None:
        raise SBMLError("no <model>")
    for unsupported in ("listOfEvents", "listOfRules", "listOfFunctionDefinitions",
                        "listOfInitialAssignments", "listOfConstraints"):
        lst = _child(model, unsupported)
        if lst is not None and len(lst):
            raise SBMLError(f"<{unsupported}> is not supported")

    symbols: Dict[str, float] = {}
    for comp in _items(model, "listOfCompartments", "compartment"):
        size = comp.get("size", comp.get("volume", "1"))
        symbols[comp.get("id")] = float(size)
    for par in _items(model, "listOfParameters", "parameter"):
        if par.get("value") is None:
            raise SBMLError(f"parameter '{par.get('id')}' has no value")
        symbols[par.get("id")] = float(par.get("value"))

    state: List[str] = []      # species that change, in document order
    fixed: Dict[str, int] = {}  # boundary / constant species and their counts
    init: Dict[str, int] = {}
    for sp in _items(model, "listOfSpecies", "species"):
        sid = sp.get("id")
        amount = sp.get("initialAmount", sp.get("initialConcentration", "0"))
        f = float(amount)
        if f != int(f) or f < 0:
            raise SBMLError(f"species '{sid}': initial amount {amount} is not a count")
        init[sid] = int(f)
        if sp.get("boundaryCondition") == "true" or sp.get("constant") == "true":
            fixed[sid] = int(f)
        else:
            state.append(sid)
    all_species = set(state) | set(fixed)
    index = {s: i for i, s in enumerate(state)}

    rxns = []   # (reactants {state idx: m}, products {state idx: m}, theta, id)
    for rx in _items(model, "listOfReactions", "reaction"):
        rid = rx.get("id")
        where = f"reaction '{rid}'"
        reac: Dict[str, int] = {}
        prod: Dict[str, int] = {}
        for ref in _items(rx, "listOfReactants", "speciesReference"):
            reac[ref.get("species")] = reac.get(ref.get("species"), 0) + _int_stoich(ref, where)
        for ref in _items(rx, "listOfProducts", "speciesReference"):
            prod[ref.get("species")] = prod.get(ref.get("species"), 0) + _int_stoich(ref, where)
        mods = [m.get("species") for m in
                _items(rx, "listOfModifiers", "modifierSpeciesReference")]
        for s in list(reac) + list(prod) + mods:
            if s not in all_species:
                raise SBMLError(f"{where}: unknown species '{s}'")
        law = _child(rx, "kineticLaw")
        if law is None:
            raise SBMLError(f"{where}: no kinetic law")
        local = dict(symbols)
        for lname in ("listOfLocalParameters", "listOfParameters"):
            for par in _items(law, lname, "localParameter") + _items(law, lname, "parameter"):
                local[par.get("id")] = float(par.get("value"))
        math_el = _child(law, "math")
        if math_el is None:
            raise SBMLError(f"{where}: kinetic law without MathML")
        terms = _eval(math_el, local, all_species, where)
        # a modifier that appears in the forward law with power e is a catalyst: reactant
        # and product with multiplicity e
        for m in mods:
            e = terms[0][1].get(m, 0)
            if e and m not in reac:
                reac[m] = e
                prod[m] = prod.get(m, 0) + e
        sides = [(reac, prod, terms[0], rid)]
        if len(terms) == 2:
            if rx.get("reversible") == "false":
                raise SBMLError(f"{where}: a difference law on an irreversible reaction")
            c, p = terms[1]
            sides.append((prod, reac, (-c, p), rid + "_reverse"))
        for re_, pr_, (coef, powers), name in sides:
            if powers != {s: m for s, m in re_.items() if m > 0}:
                raise SBMLError(f"reaction '{name}': law species {powers} do not match the "
                                f"reactants {re_} (not mass action)")
            if not (coef >= 0.0) or not math.isfinite(coef):
                raise SBMLError(f"reaction '{name}': rate constant {coef} is not >= 0")
            theta = coef
            rr: Dict[int, int] = {}
            pp: Dict[int, int] = {}
            for s, m in re_.items():
                if s in fixed:
                    theta *= math.comb(fixed[s], m)
                elif m:
                    rr[index[s]] = m
            for s, m in pr_.items():
                if s not in fixed and m:
                    pp[index[s]] = m
            if any(m > 3 for m in rr.values()):
                raise SBMLError(f"reaction '{name}': reactant order above 3")
            rxns.append((rr, pp, theta, name))

    if not state:
        raise SBMLError("no species that can change")
    if not rxns:
        raise SBMLError("no reactions")
    M, N = len(rxns), len(state)
    orders = np.zeros((M, N), np.int32)
    stoich = np.zeros((M, N), np.int32)
    rates = np.zeros(M)
    for j, (rr, pp, theta, _) in enumerate(rxns):
        for s, m in rr.items():
            orders[j, s] = m
            stoich[j, s] -= m
        for s, m in pp.items():
            stoich[j, s] += m
        rates[j] = theta
    name = model.get("id") or model.get("name") or "sbml_model"
    crn = CRN(name, orders, stoich, rates, tuple(state))
    x0 = np.array([init[s] for s in state], np.int64)
    return SBMLModel(crn, x0, tuple(r[3] for r in rxns))


def load_sbml(path: str) -> SBMLModel:
    with open(path, "r", encoding="utf-8") as f:
        return read_sbml(f.read())


def write_sbml(crn: CRN, x0, model_id: str = None) -> str:
    """SBML Level 3 Version 1 core text for a mass-action CRN: one compartment of size 1,
    species with initial amounts x0, one parameter per reaction and the law
    k_j * prod_s S_s^m_js (read back by read_sbml to the same arrays)."""
    x0 = np.asarray(x0, np.int64).reshape(-1)
    N, M = crn.n_species, crn.n_reactions
    names = list(crn.species) if len(crn.species) == N else [f"S{s}" for s in range(N)]
    mid = model_id or crn.name
    out = ['<?xml version="1.0" encoding="UTF-8"?>',
           '<sbml xmlns="http://www.sbml.org/sbml/level3/version1/core" level="3" version="1">',
           f'  <model id="{mid}">',
           '    <listOfCompartments>',
           '      <compartment id="cell" size="1" constant="true" spatialDimensions="3"/>',
           '    </listOfCompartments>', '    <listOfSpecies>']
    for s in range(N):
        out.append(f'      <species id="{names[s]}" compartment="cell" initialAmount="{int(x0[s])}" '
                   'hasOnlySubstanceUnits="true" boundaryCondition="false" constant="false"/>')
    out += ['    </listOfSpecies>', '    <listOfParameters>']
    for j in range(M):
        out.append(f'      <parameter id="k{j}" value="{float(crn.rates[j])!r}" constant="true"/>')
    out += ['    </listOfParameters>', '    <listOfReactions>']
    for j in range(M):
        out.append(f'      <reaction id="R{j}" reversible="false">')
        reac = [(s, int(crn.orders[j, s])) for s in range(N) if crn.orders[j, s] > 0]
        prod = [(s, int(crn.orders[j, s] + crn.stoich[j, s])) for s in range(N)
                if crn.orders[j, s] + crn.stoich[j, s] > 0]
        for tag, lst in (("listOfReactants", reac), ("listOfProducts", prod)):
            if lst:
                out.append(f'        <{tag}>')
                for s, m in lst:
                    out.append(f'          <speciesReference species="{names[s]}" '
                               f'stoichiometry="{m}" constant="true"/>')
                out.append(f'        </{tag}>')
        factors = [f'<ci>k{j}</ci>']
        for s, m in reac:
            factors.append(f'<ci>{names[s]}</ci>' if m == 1 else
                           f'<apply><power/><ci>{names[s]}</ci><cn type="integer">{m}</cn></apply>')
        body = factors[0] if len(factors) == 1 else '<apply><times/>' + ''.join(factors) + '</apply>'
        out += ['        <kineticLaw>',
                f'          <math xmlns="http://www.w3.org/1998/Math/MathML">{body}</math>',
                '        </kineticLaw>', '      </reaction>']
    out += ['    </listOfReactions>', '  </model>', '</sbml>', '']
    return "\n".join(out)
