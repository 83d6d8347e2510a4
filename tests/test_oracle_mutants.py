"""Planted mistakes: each mutant of the oracle source must fail at least one pin.

The mutations are applied to a copy of oracle/cf_oracle.c in a temporary directory and
compiled there (CPU only); the oracle itself is never modified.  This shows that the pins
in test_oracle_pins.py constrain every part of the oracle a plausible mistake could touch:
the separation, the periodic wrap, the bin edges, the doubling and self pairs of
auto-correlations (their counts and their weights), the pi cut, the rp/pi split, angular edges,
weights and ravg (of r, of rp for DD(rp, pi) and wp, and of rp for the mocks).
"""
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
from tests.test_oracle_mocks import MOCK_CHECKS
from tests.test_oracle_pins import LATTICE, PERIODIC, RPPI, Cat

MUTANTS = {
    # observed / mock galaxies (Appendix A.2.1)
    "mocks_los_from_difference": ("double lx = 0.5 * (xi + xj)", "double lx = 0.5 * (xi - xj)"),
    "mocks_pi_not_normalised": ("double pi2 = ll > 0.0 ? (sl * sl) / ll : 0.0;",
                                "double pi2 = ll > 0.0 ? (sl * sl) : 0.0;"),
    "mocks_rp_adds_pi": ("double rp2 = ss - pi2;", "double rp2 = ss + pi2;"),
    "mocks_pi_edges_unsquared": ("or_find(p->pe2, p->npi, pi2)", "or_find(p->pe, p->npi, pi2)"),
    "mocks_drop_sz_term": ("ss = ss + sz * sz;", "ss = ss;"),
    "mocks_pimax_inclusive": ("if (!(pi2 < p->pimax2)) return -1;", "if (!(pi2 <= p->pimax2)) return -1;"),
    "drop_dz_term": ("s = s + dz * dz;", "s = s;"),
    "wrap_wrong_sign": ("if (d > 0.5 * L) d -= L;", "if (d > 0.5 * L) d += L;"),
    "lower_edge_exclusive": ("if (s < p->e2[0] || s >= p->e2[nb]) return -1;\n        int k",
                             "if (s <= p->e2[0] || s >= p->e2[nb]) return -1;\n        int k"),
    "upper_edge_inclusive": ("if (s < p->e2[0] || s >= p->e2[nb]) return -1;\n        int k",
                             "if (s < p->e2[0] || s > p->e2[nb]) return -1;\n        int k"),
    "ties_to_lower_bin": ("while (k > 0 && s < e[k]) k--;", "while (k > 0 && s <= e[k]) k--;"),
    "no_auto_doubling": ("npairs[k] *= 2; wsum[k] *= 2.0; rsum[k] *= 2.0;", ""),
    "no_self_pairs": ("npairs[k] += (uint64_t)n1;", ""),
    "pimax_inclusive": ("if (!(pi < p->pimax)) return -1;", "if (!(pi <= p->pimax)) return -1;"),
    "rp_uses_dz": ("double s = dx * dx + dy * dy;\n    double pi = fabs(dz);",
                   "double s = dx * dx + dz * dz;\n    double pi = fabs(dz);"),
    "pi_uses_dy": ("double pi = fabs(dz);", "double pi = fabs(dy);"),
    "rppi_index_transposed": ("return k * p->npi + m;", "return m * p->nbins + k;"),
    "theta_full_angle": ("double c = 2.0 * sin(e * (M_PI / 360.0));\n            p->e2[k] = c * c;\n        } else {\n            p->e2[k] = e * e;\n        }\n    }\n    p->npi",
                         "double c = 2.0 * sin(e * (M_PI / 180.0));\n            p->e2[k] = c * c;\n        } else {\n            p->e2[k] = e * e;\n        }\n    }\n    p->npi"),
    "weight_sum_not_product": ("double ww = wi * (w2 ? w2[j] : 1.0);", "double ww = wi + (w2 ? w2[j] : 1.0);"),
    "ravg_squared": ("double c = sqrt(s);", "double c = s;"),
    "rppi_ravg_3d_separation": ("if (p->ravg) *sep = sqrt(s);\n    if (p->kind == OR_WP) return k;",
                                "if (p->ravg) *sep = sqrt(s + dz * dz);\n    if (p->kind == OR_WP) return k;"),
    "mocks_ravg_3d_separation": ("if (p->ravg) *sep = sqrt(rp2);", "if (p->ravg) *sep = sqrt(ss);"),
    "mocks_ravg_is_pi": ("if (p->ravg) *sep = sqrt(rp2);", "if (p->ravg) *sep = sqrt(pi2);"),
    "ravg_ignores_weights": ("if (P.ravg) hr[k] += (P.weighted ? ww : 1.0) * sep;", "if (P.ravg) hr[k] += sep;"),
    "no_self_pair_weights": ("wsum[k] += sw;", ""),
    "self_pair_weight_is_one": ("sw += w1 ? w1[i] * w1[i] : 1.0;", "sw += 1.0;"),
    "self_pair_weight_not_squared": ("sw += w1 ? w1[i] * w1[i] : 1.0;", "sw += w1 ? w1[i] : 1.0;"),
    "rows_self_pair_weight_is_one": ("if (k >= 0) { hc[k] += 1; hw[k] += wi * wi; }",
                                     "if (k >= 0) { hc[k] += 1; hw[k] += 1.0; }"),
    "cross_skips_first_row": ("ra[0] = (rowwise || !autoc) ? 0 : i + 1;",
                              "ra[0] = (rowwise || !autoc) ? 1 : i + 1;"),
}


def _pin_checks(lib):
    """The quick pins, each returning normally or raising AssertionError."""
    import gen

    def lattice():
        out = oracle.count("r", [1, 2, 3, 5, 6], Cat(LATTICE), autocorr=True, periodic=False,
                           mode="brute", lib=lib)
        assert out["npairs"].tolist() == [2, 4, 4, 2]

    def lattice_w():
        d = Cat(LATTICE, w=[1.0, 2.0, 0.5, 4.0])
        out = oracle.count("r", [1, 2, 3, 5, 6], d, autocorr=True, periodic=False, weighted=True,
                           ravg=True, mode="brute", lib=lib)
        assert out["wsum"].tolist() == [4.0, 3.0, 20.0, 8.0]
        exp = [1.0, (0.5 * 2 + math.sqrt(5)) / 1.5, (8 * math.sqrt(20) + 2 * math.sqrt(13)) / 10, 5.0]
        np.testing.assert_allclose(out["ravg"], exp, rtol=1e-15)

    def periodic():
        d = Cat(PERIODIC)
        out = oracle.count("r", [0, 1, 2, 4, 5], d, autocorr=True, periodic=True, box=8.0,
                           mode="brute", lib=lib)
        assert out["npairs"].tolist() == [7, 4, 2, 10]
        out = oracle.count("r", [0, 1, 2, 4, 5], d, d, autocorr=False, periodic=True, box=8.0,
                           mode="brute", lib=lib)
        assert out["npairs"].tolist() == [7, 4, 2, 10]

    def rppi():
        out = oracle.count("rppi", [1, 2, 3, 5, 6], Cat(RPPI), autocorr=True, periodic=False,
                           pimax=3.0, npibins=3, mode="brute", lib=lib)
        exp = np.zeros((4, 3), dtype=np.uint64)
        exp[0, 1], exp[1, 0], exp[2, 2] = 2, 4, 4
        assert (out["npairs"] == exp).all()

    def rppi_ravg():
        from tests.test_oracle_pins import RPPI_W
        kw = dict(autocorr=True, periodic=False, pimax=3.0, npibins=3, mode="brute", lib=lib, ravg=True)
        out = oracle.count("rppi", [1, 2, 3, 5, 6], Cat(RPPI), **kw)
        np.testing.assert_allclose(out["ravg"][0, 1], 1.0, rtol=1e-15)
        np.testing.assert_allclose(out["ravg"][1, 0], (2 + math.sqrt(5)) / 2, rtol=1e-15)
        wp = oracle.count("wp", [1, 2, 3, 5, 6], Cat(RPPI, w=RPPI_W), weighted=True, **kw)
        np.testing.assert_allclose(wp["ravg"][:3], [1.0, (1 + math.sqrt(5)) / 1.5,
                                                   (8 * math.sqrt(20) + 2 * math.sqrt(13)) / 10], rtol=1e-15)

    def self_pair_weights():
        from tests.test_oracle_pins import PERIODIC_W
        d = Cat(PERIODIC, w=PERIODIC_W)
        kw = dict(periodic=True, box=8.0, weighted=True, ravg=True, autocorr=True, lib=lib)
        for out in (oracle.count("r", [0, 2, 4, 5], d, mode="brute", **kw),
                    oracle.count("r", [0, 2, 4, 5], d, rows=(0, 5), **kw)):
            assert out["wsum"].tolist() == [34.3125, 2.0, 23.5]
            np.testing.assert_allclose(out["ravg"][0], 5.0 / 34.3125, rtol=1e-15)

    def theta():
        d = Cat([(1, 0, 0), (0, 1, 0), (0, 0, 1), (-1, 0, 0)])
        out = oracle.count("theta", [60, 90, 180], d, autocorr=True, periodic=False, mode="brute",
                           lib=lib)
        assert out["npairs"].tolist() == [0, 10]

    def totals():
        d = gen.uniform_box(200, 10.0, 51)
        e = gen.uniform_box(150, 10.0, 52)
        out = oracle.count("r", [1e-6, 9.0], d, e, autocorr=False, periodic=True, box=10.0, lib=lib)
        assert int(out["npairs"].sum()) == d.n * e.n

    def ckdtree():
        from scipy.spatial import cKDTree
        d = gen.uniform_box(800, 30.0, 11, dtype=np.float64)
        edges = gen.log_edges(0.5, 10.0, 6)
        out = oracle.count("r", edges, d, autocorr=True, periodic=True, box=30.0, mode="brute", lib=lib)
        a = np.stack([d.x, d.y, d.z], 1)
        t = cKDTree(a, boxsize=30.0)
        assert out["npairs"].astype(np.int64).tolist() == np.diff(t.count_neighbors(t, edges)).astype(np.int64).tolist()

    mocks = []
    for chk in MOCK_CHECKS:
        def run(chk=chk):
            chk(lib)
        run.__name__ = chk.__name__
        mocks.append(run)
    return [lattice, lattice_w, periodic, rppi, rppi_ravg, self_pair_weights, theta, totals, ckdtree] + mocks


def _build_mutant(tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "cf_oracle.c")).read()
    assert src.count(old) >= 1, f"mutation {name} does not apply"
    mutated = src.replace(old, new, 1)
    c = tmp_path / f"{name}.c"
    c.write_text(mutated)
    so = tmp_path / f"{name}.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", str(c),
                    "-o", str(so), "-lm"], check=True)
    return oracle.load(str(so))


def test_unmutated_passes_all_pins(orc):
    for chk in _pin_checks(orc):
        chk()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    pytest.importorskip("scipy.spatial")
    old, new = MUTANTS[name]
    lib = _build_mutant(tmp_path, name, old, new)
    failed = []
    for chk in _pin_checks(lib):
        try:
            chk()
        except AssertionError:
            failed.append(chk.__name__)
    assert failed, f"mutant {name} passed every pin"
