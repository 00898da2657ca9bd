"""Planted mistakes: each one is written into a copy of the oracle's C source,
compiled on the CPU, loaded in place of the oracle for the duration of one
pin, and must make that pin fail.  This shows the pins catch the mistakes a
restatement of the paper is likely to make (a sign, a dropped term, an index,
an exponent, an offset)."""
import contextlib
import subprocess

import pytest

from oracle import api as orc_api

import test_oracle_codec as tcodec
import test_oracle_counts as tcounts
import test_oracle_keys as tkeys
import test_oracle_learned_inputs as tlearn
import test_oracle_neighbors as tneigh
import test_oracle_sph as tsph


@contextlib.contextmanager
def _mutant(tmp_path, old, new):
    src = open(orc_api._SRC).read()
    assert src.count(old) == 1, old
    msrc = tmp_path / "nl_oracle.c"
    msrc.write_text(src.replace(old, new))
    out = tmp_path / "liboracle.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
                           "-fno-fast-math", "-shared", "-fPIC", "-o", str(out), str(msrc), "-lm"])
    saved = (orc_api._OUT, orc_api._SRC, orc_api._lib)
    with orc_api._lock:
        orc_api._OUT, orc_api._SRC, orc_api._lib = str(out), str(msrc), None
    try:
        yield
    finally:
        with orc_api._lock:
            orc_api._OUT, orc_api._SRC, orc_api._lib = saved


MUTANTS = [
    ("periodic wrap sign",
     "        if (d32 > half) d -= (double)len;",
     "        if (d32 > half) d += (double)len;",
     lambda orc: tsph.test_ljc_periodic_minimum_image(orc)),
    ("Coulomb sign",
     "if (q) c += kc * (double)q[i] * (double)q[j] / (r2 * r);",
     "if (q) c -= kc * (double)q[i] * (double)q[j] / (r2 * r);",
     lambda orc: tsph.test_ljc_two_particles_closed_forms(orc)),
    ("density self term dropped",
     "double s = (double)ms[i] * orc_W(0.0, h);",
     "double s = 0.0;",
     lambda orc: tsph.test_density_against_direct_sum(orc)),
    ("kernel normalisation h^2 instead of h^3",
     "return orc_w(r / h) / (M_PI * h * h * h);",
     "return orc_w(r / h) / (M_PI * h * h);",
     lambda orc: tsph.test_kernel_normalisation_and_shape(orc)),
    ("pressure-force gradient of h_j with h^3",
     "double gj = orc_dw(r / hj) / (M_PI * hj * hj * hj * hj);",
     "double gj = orc_dw(r / hj) / (M_PI * hj * hj * hj);",
     lambda orc: tsph.test_pressure_force_is_minus_energy_gradient(orc)),
    ("LJ force exponent",
     "double r4 = r2 * r2, r8 = r4 * r4, r14 = r8 * r4 * r2;\n"
     "            double c = 24.0 * eps * (2.0 * s12 / r14 - s6 / r8);\n"
     "            ax += c * (-dx);",
     "double r4 = r2 * r2, r8 = r4 * r4, r14 = r8 * r4 * r2;\n"
     "            double c = 24.0 * eps * (2.0 * s12 / r14 - s6 / r14);\n"
     "            ax += c * (-dx);",
     lambda orc: tsph.test_lj_force_energy_and_newton3(orc)),
    ("codec info nibble offset",
     "info[ni++] = (uint8_t)(v + 6);",
     "info[ni++] = (uint8_t)(v + 5);",
     lambda orc: tcodec.test_table1_worked_examples(orc)),
    ("Morton bit order",
     "key = (key << 3) | ((uint64_t)((qx >> b) & 1u) << 2) |\n"
     "              ((uint64_t)((qy >> b) & 1u) << 1) | (uint64_t)((qz >> b) & 1u);",
     "key = (key << 3) | ((uint64_t)((qy >> b) & 1u) << 2) |\n"
     "              ((uint64_t)((qx >> b) & 1u) << 1) | (uint64_t)((qz >> b) & 1u);",
     lambda orc: tkeys.test_morton_closed_form(orc)),
    ("Hilbert Gray step dropped",
     "for (int i = 1; i < 3; ++i) X[i] ^= X[i - 1];",
     "for (int i = 2; i < 3; ++i) X[i] ^= X[i - 1];",
     lambda orc: tkeys.test_hilbert_bijection_and_adjacency(orc, 3)),
    ("sort ties reversed",
     "if (u->idx != v->idx) return u->idx < v->idx ? -1 : 1;",
     "if (u->idx != v->idx) return u->idx < v->idx ? 1 : -1;",
     lambda orc: tkeys.test_sort_is_stable_by_original_index(orc)),
    ("feature window of 8 super-clusters shifted by one",
     "for (int64_t t = s - 3; t < s + 5; ++t)",
     "for (int64_t t = s - 4; t < s + 4; ++t)",
     lambda orc: tlearn.test_region_features_of_a_line_of_super_clusters(orc)),
    ("feature length floor dropped",
     "return e > floor_len ? e : floor_len;",
     "return e;",
     lambda orc: tlearn.test_features_of_hand_built_system(orc)),
    ("target mean over the cluster's M slots instead of its real particles",
     "y[c] = k ? log(s / (double)k / e64[c / 8]) : 0.0;",
     "y[c] = k ? log(s / (double)M / e64[c / 8]) : 0.0;",
     lambda orc: tlearn.test_targets_of_hand_built_system(orc)),
    ("h at count between the (k+1)-th and (k+2)-th neighbor",
     "float dk1 = hp[0], dk = hp[1];",
     "float dk1 = hp[0] * 1.5f, dk = hp[0];",
     lambda orc: tcounts.test_h_at_count_has_exactly_k_neighbors(orc, "uniform", 40)),
    ("computed pairs count M x M for M x MJ tiles",
     "return s * (int64_t)cluster * (int64_t)jcluster;",
     "return s * (int64_t)cluster * (int64_t)cluster;",
     lambda orc: tcounts.test_computed_pairs_all_in_range_and_isolated(orc, 8, 4)),
    ("nearest keeps the largest distance",
     "if (r < best) best = r;",
     "if (r > best || best == INFINITY) best = r;",
     lambda orc: tneigh.test_nearest_distance_against_kd_tree(orc, "uniform")),
]


@pytest.mark.parametrize("name,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_its_pin(tmp_path, orc, name, old, new, pin):
    # the pin passes on the oracle itself
    pin(orc)
    with _mutant(tmp_path, old, new):
        with pytest.raises(AssertionError):
            pin(orc)
    # and again after the oracle is back
    pin(orc)


def test_planted_mistake_in_the_half_list_filter(orc, monkeypatch):
    """The half-list definition with the super-cluster's own first cluster
    left out fails the half-list pin."""
    import inspect

    import oracle
    src = inspect.getsource(orc_api.half_lists)
    assert src.count("Js >= 8 * s") == 1
    ns = dict(orc_api.__dict__)
    exec(compile(src.replace("Js >= 8 * s", "Js > 8 * s"), "half_lists_mutant", "exec"), ns)
    tneigh.test_half_lists_store_every_cluster_pair_once(orc, "uniform", 8)
    monkeypatch.setattr(oracle, "half_lists", ns["half_lists"])
    with pytest.raises(AssertionError):
        tneigh.test_half_lists_store_every_cluster_pair_once(orc, "uniform", 8)
