"""Planted mistakes in the oracle fail its pins.

Each case copies the oracle's C source, replaces one expression by a plausible mistake
(a dropped term or factor, a flipped sign, an index off by one, a transposed operand,
swapped operands, a reversed comparison), compiles the copy with the oracle's own flags
into a temporary library, routes the oracle module to it and runs pins of
tests/test_oracle_*.py against it, cheapest first: at least one must fail.  The
unmodified source, copied and compiled the same way, passes every pin of the list, so a
failure comes from the planted mistake and not from the harness.

Every planted mistake keeps all memory accesses inside their arrays (an index moved by
one stays within the same table; a transposed index ranges over the same elements)."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
import test_oracle_codes as codes_pins
import test_oracle_compact as compact_pins
import test_oracle_constants as const_pins
import test_oracle_frameq as frameq_pins
import test_oracle_hier as hier_pins
import test_oracle_permutation as perm_pins
import test_oracle_precision as prec_pins
import test_oracle_rng as rng_pins
import test_oracle_routing_test as routing_pins
import test_oracle_search as search_pins
import test_oracle_simhash as sh_pins
import workloads
from workloads.graph import build_graph
from workloads.hier import build_hierarchy

SRC = os.path.join(os.path.dirname(oracle.__file__), "peos_oracle.c")

# (name, passage the expression restates, original text, planted text)
MUTATIONS = [
    ("x not normalised", "Sec. 4.2 step (5): the table is of x / ||x||",
     "tmp[k] = y[k] / yn;", "tmp[k] = y[k];"),
    ("sign of H_2 flipped", "Eq. (combination): + sgn(e[0]) x'.b",
     "float h2 = (c0 > 0) ? t[j0] : -t[j0];", "float h2 = (c0 > 0) ? -t[j0] : t[j0];"),
    ("H_1 reads the previous block's table", "Sec. 4.2 step (5): block i of x against a^i",
     "float tv = t[(size_t)i * m + j];", "float tv = t[(size_t)(i - 1) * m + j];"),
    ("A^2 term of the variance dropped", "Eq. (N_ex_min): var = w_reg^2 + L w_res^2 - L A^2 / (L + 1)",
     "float var = (wr * wr + cr * cr) - (Lf * (A * A)) / (Lf + 1.0f);", "float var = (wr * wr + cr * cr);"),
    ("quantile taken above the mean", "Eq. (LB): T = A c + Phi^{-1}(eps) sqrt(var), Phi^{-1}(eps) < 0",
     "return A * P->c_eta + P->z_eps * sqrtf(fmaxf(var, 0.0f));",
     "return A * P->c_eta - P->z_eps * sqrtf(fmaxf(var, 0.0f));"),
    ("decision reversed", "Algorithm 2: pass iff H >= T",
     "r.pass = (r.H - r.T) >= 0.0f;", "r.pass = (r.T - r.H) >= 0.0f;"),
    ("factor 2 of A dropped", "Eq. (A_r) translated by -v: A = (|x|^2 + |e|^2 - delta^2) / (2 |x| |e|)",
     "float A = ((dv + en * en) - delta2) / (2.0f * (xn * en));", "float A = ((dv + en * en) - delta2) / (xn * en);"),
    ("sign of r in frame Q's A_r", "Eq. (A_r): A_r = (|u|^2 / 2 - r - v.q) / (|q| |e|)",
     "float A = ((un2 / 2.0f - r_) - vq) / (qn * en);", "float A = ((un2 / 2.0f + r_) - vq) / (qn * en);"),
    ("x = v - q in the search", "frame translated by -v: x = q - v",
     "for (int k = 0; k < d; ++k) xv[k] = qi[k] - vrow[k];", "for (int k = 0; k < d; ++k) xv[k] = vrow[k] - qi[k];"),
    ("x = v - q in the edge statistics", "frame translated by -v: x = q - v",
     "for (int k = 0; k < d; ++k) xv[k] = qi[k] - Xi[(size_t)v * d + k];",
     "for (int k = 0; k < d; ++k) xv[k] = Xi[(size_t)v * d + k] - qi[k];"),
    ("projection block transposed", "Algorithm 2's table: t[i][j] = x_i . a^i_j",
     "const float* a = A + ((size_t)i * m + j) * dp;\n      float acc = 0.0f;\n"
     "      for (int k = 0; k < dp; ++k) acc = acc + a[k] * x[i * dp + k];",
     "const float* a = A + ((size_t)j * L + i) * dp;\n      float acc = 0.0f;\n"
     "      for (int k = 0; k < dp; ++k) acc = acc + a[k] * x[i * dp + k];"),
    ("sqrt(L) of w_reg dropped", "Sec. 4.2 step (1): w_reg = sum_i |e_i| / (sqrt(L) |e|)",
     "float w = s / (sqrtf((float)L) * en);", "float w = s / en;"),
    ("residual coefficient inverted", "Sec. 4.2 step (1): e_res = e - e_reg, block i scaled by 1 - mean|e_k| / |e_i|",
     "(1.0f - mean_bn / bn[i])", "(1.0f - bn[i] / mean_bn)"),
    ("sign of the block codes dropped", "Sec. 4.2 step (3): e[i] = sgn * argmax_j |e_i . a^i_j|",
     "codes[i + 1] = (int8_t)((p[jb] >= 0.0f) ? (jb + 1) : -(jb + 1));", "codes[i + 1] = (int8_t)(jb + 1);"),
    ("eta of ln m", "Lemma 4.2: eta = sqrt(2 ln m)",
     "if (mode == 0) return sqrt(2.0 * log((double)m));", "if (mode == 0) return sqrt(log((double)m));"),
    ("Box-Muller pair both cosines", "Sec. 4.2 step (2): independent N(0, 1) draws",
     "z[2 * h + 1] = r * sin(th);", "z[2 * h + 1] = r * cos(th);"),
    ("Philox key schedule", "Philox4x64-10 (Salmon et al.): Weyl constants of the key schedule",
     "k1 += PHILOX_W1;", "k1 += PHILOX_W0;"),
    ("squared distance without the square", "Sec. 2: squared l2 distance",
     "{ float t = a[k] - b[k]; acc = acc + t * t; }", "{ float t = a[k] - b[k]; acc = acc + fabsf(t); }"),
    ("list bound from the first entry", "Algorithm 1: delta = the efs-th distance of R",
     "float delta2 = full ? R[ef - 1].dist : INFINITY;", "float delta2 = full ? R[0].dist : INFINITY;"),
    ("insertion accepts a tie with the bound", "Algorithm 1: insert iff dist < delta",
     "if (*len == ef && !(dist < R[ef - 1].dist)) return 0;", "if (*len == ef && !(dist <= R[ef - 1].dist)) return 0;"),
    ("quantile table bin's lower edge", "Sec. 4.3: the bin's bound keeps the quantile below the true one",
     "return (float)(bin + 1) * (1.0f / 256.0f);", "return (float)(bin) * (1.0f / 256.0f);"),
    ("visited marked before the test", "Sec. 3.1's remedy: a neighbour that fails can pass later from another node",
     "if (vs->seen[u]) { cnt[C_VISITED_SKIP]++; continue; }",
     "if (vs->seen[u]) { cnt[C_VISITED_SKIP]++; continue; }\n        if (!vis_mark(vs, u)) return ORC_E_NOMEM;"),
    ("frame Q's v.q from the bound's node", "Eq. (A_r): v.q of the expanded node",
     "vq = dot_f32(ix->X + (size_t)v * d, q, d);", "vq = dot_f32(ix->X + (size_t)R[ef - 1].id * d, q, d);"),
    ("re-rank without sorting again", "the precision form: the final list re-ranked in exact FP32",
     "          qsort(Rl, (size_t)len, sizeof(rentry), cmp_cand);\n", ""),
    ("per-query entries ignored", "the hierarchical entry: each query starts at its own node",
     "entries ? entries[qi] : entry", "entry"),
    ("BF16 rounds half up", "round to nearest, ties to even",
     "u += 0x7fffu + lsb;", "u += 0x8000u;"),
    ("E4M3 ties round down", "round to nearest, ties to even",
     "int best = (dl < dh) ? lo : (dh < dl) ? hi : ((lo & 1) == 0 ? lo : hi);",
     "int best = (dl < dh) ? lo : (dh < dl) ? hi : lo;"),
    ("E4M3 subnormal exponent", "E4M3: subnormals m / 8 * 2^-6",
     "ldexpf((float)man / 8.0f, -6)", "ldexpf((float)man / 8.0f, -7)"),
    ("E4M3 scale constant", "per-row scale max|x| / 448",
     "float sc = amax > 0.0f ? amax / 448.0f : 1.0f;", "float sc = amax > 0.0f ? amax / 240.0f : 1.0f;"),
    ("compact range one step wide", "Sec. 4.3: b-bit signed integers, |q| <= 2^(b-1) - 1",
     "const float Qb = (float)((1 << (bits - 1)) - 1);", "const float Qb = (float)(1 << (bits - 1));"),
    ("compact rounding down", "round to nearest, ties to even",
     "float r = rintf(x[s] / step);", "float r = floorf(x[s] / step);"),
    ("permutation serves the lightest subspace", "Appendix D.1: the subspace with the greatest running sum",
     "(best < 0 || load[i] > load[best])", "(best < 0 || load[i] < load[best])"),
    ("permutation order descending", "Appendix D.1: coordinates in ascending Avg(e_j^2)",
     "if (x->v < y->v) return -1;\n  if (x->v > y->v) return 1;", "if (x->v < y->v) return 1;\n  if (x->v > y->v) return -1;"),
    ("Hoeffding margin subtracted", "Sec. 3.1: P(#Col <= K p - t) <= exp(-2 t^2 / K)",
     "const double r = ((double)c + t) / (double)K;", "const double r = ((double)c - t) / (double)K;"),
    ("SimHash differences counted as collisions", "Lemma 4.1: #Col = K - Hamming distance",
     "const int col = sh->K - diff;", "const int col = diff;"),
    ("descent ties keep the higher id", "the hierarchical entry's (dist, id) order",
     "(du == db && ids[u] < ids[best])", "(du == db && ids[u] > ids[best])"),
    ("pruning rule inverted", "relative-neighbourhood pruning: drop c if a kept s is closer to c than x is",
     "X + (size_t)cand[c].id * d, d) < cand[c].dist)", "X + (size_t)cand[c].id * d, d) > cand[c].dist)"),
    ("degenerate edges rejected", "a zero edge (duplicate vectors) or q = v always passes",
     "{ r.kind = 3; return r; }", "{ r.kind = 3; r.pass = 0; return r; }"),
    ("A >= 1 accepted", "Algorithm 2: A >= 1 rejects",
     "if (A >= 1.0f) { r.pass = 0; r.kind = 0; return r; }", "if (A >= 1.0f) { r.pass = 1; r.kind = 0; return r; }"),
    ("A <= 0 rejected", "Algorithm 2: A <= 0 accepts",
     "if (A <= 0.0f) { r.pass = 1; r.kind = 1; return r; }", "if (A <= 0.0f) { r.pass = 0; r.kind = 1; return r; }"),
    ("e[0] from e instead of e_res", "Sec. 4.2 step (3): e[0] = argmax_j |e_res . b_j|",
     "for (int k = 0; k < d; ++k) acc = acc + b[k] * eres[k];", "for (int k = 0; k < d; ++k) acc = acc + b[k] * e[k];"),
    ("query not permuted", "Appendix D.1: the query is read in the permuted coordinates",
     "qi[t] = perm ? q[perm[t]] : q[t];", "qi[t] = q[t];"),
    ("frame Q's |q| without the square root", "Algorithm 2: the table of q' = q / ||q||",
     "qn = sqrtf(dot_f32(q, q, d));", "qn = dot_f32(q, q, d);"),
    ("SimHash bits of x complemented", "Sec. 3.1: bit i of x is [S_i . x >= 0]",
     "if (dot_f32(sh->S + (size_t)i * d, xv, d) >= 0.0f)", "if (dot_f32(sh->S + (size_t)i * d, xv, d) < 0.0f)"),
    ("brute-force ties by descending id", "Sec. 2's K-NN with ties taken in id order",
     "while (pos > 0 && (dist < top[pos - 1].dist || (dist == top[pos - 1].dist && id < top[pos - 1].id)))",
     "while (pos > 0 && (dist < top[pos - 1].dist || (dist == top[pos - 1].dist && id > top[pos - 1].id)))"),
    ("empty result slots at distance 0", "an empty slot of the output is (-1, +inf)",
     "dists_out[(size_t)qi * P->k + j] = j < len ? Rl[j].dist : INFINITY;",
     "dists_out[(size_t)qi * P->k + j] = j < len ? Rl[j].dist : 0.0f;"),
    ("lazy codes from the searched rows", "the index is built from the FP32 rows",
     "build_node(ix->Xi, ix->d,", "build_node(ix->X, ix->d,"),
    ("re-rank from the searched rows", "the precision form: the re-rank reads the FP32 rows",
     "Rl[j].dist = orc_dist2_f32(q, Xr + (size_t)Rl[j].id * d, d);",
     "Rl[j].dist = orc_dist2_f32(q, ix.X + (size_t)Rl[j].id * d, d);"),
    ("E4M3 saturates to the NaN code", "E4M3: magnitudes beyond 448 saturate to 448",
     "return (uint8_t)((neg << 7) | 0x7e);  /* saturate to 448 */", "return (uint8_t)((neg << 7) | 0x7f);"),
    ("reverse edges dropped", "the graph: each list joined with its reverse edges, then pruned",
     "for (int64_t t = roff[y]; t < roff[y + 1]; ++t) {", "for (int64_t t = roff[y]; t < roff[y]; ++t) {"),
    ("entry not the node nearest the centroid", "the graph's entry: the node nearest the centroid",
     "if (acc < best) { best = acc; entry = (int32_t)x; }", "if (acc > best) { best = acc; entry = (int32_t)x; }"),
    ("projection counters transposed", "the generator's counter layout (column / 4, row i m + j, matrix)",
     "uint64_t row = (uint64_t)i * (uint64_t)m + (uint64_t)j;", "uint64_t row = (uint64_t)j * (uint64_t)L + (uint64_t)i;"),
]


def _small_sift():
    cfg = workloads.scaled(workloads.CONFIGS["sift"], 3000, 40)
    X, Q = workloads.generate(cfg)
    nbrs, entry = build_graph(X, 32)
    return cfg, X, Q, nbrs, entry


def _small_glove():
    cfg = workloads.scaled(workloads.CONFIGS["glove"], 4000, 40)
    X, Q = workloads.generate(cfg)
    nbrs, entry = build_graph(X, 16)
    return cfg, X, Q, nbrs, entry


def _small_simhash():
    cfg = workloads.scaled(workloads.CONFIGS["sift"], 5000, 50)
    X, Q = workloads.generate(cfg)
    nbrs, entry = build_graph(X, 16)
    return X, Q, nbrs, entry


def _small_perm():
    rng = np.random.default_rng(7)
    n, d, R = 2000, 64, 12
    scale = np.linspace(0.2, 3.0, d)[rng.permutation(d)]
    X = np.round(rng.standard_normal((n, d)) * scale * 10).astype(np.float32)
    Q = np.round(rng.standard_normal((40, d)) * scale * 10).astype(np.float32)
    nbrs, entry = build_graph(X, R)
    return X, Q, nbrs, entry


def _small_hier():
    cfg = workloads.scaled(workloads.CONFIGS["sift"], 6000, 60)
    X, Q = workloads.generate(cfg)
    nbrs, entry = build_graph(X, 16)
    layers, top = build_hierarchy(X, 16, seed=3, M=6, min_nodes=20)
    return cfg, X, Q, nbrs, entry, layers, top


def _pins(sift, glove, sift_sh, hier, perm):
    """The pins, cheapest first, as (name, callable).  Index data are built inside each
    call, so they come from the library the module is routed to."""
    def with_sift(f, *a):
        def run():
            cfg, X, Q, nbrs, entry = sift
            f((X, Q, nbrs, entry, oracle.Index(X, nbrs, entry, 8, 16, cfg.proj_seed)), *a)
        return run

    def with_glove(f):
        def run():
            cfg, X, Q, nbrs, entry = glove
            f((cfg, X, Q, nbrs, entry, oracle.Index(X, nbrs, entry, cfg.L, cfg.m, cfg.proj_seed)))
        return run

    def with_sift_q(f):
        def run():
            cfg, X, Q, nbrs, entry = sift
            f((cfg, X, Q, nbrs, entry, oracle.Index(X, nbrs, entry, cfg.L, cfg.m, cfg.proj_seed)))
        return run

    def with_sift_sh(f):
        def run():
            X, Q, nbrs, entry = sift_sh
            f((X, Q, nbrs, entry, oracle.SimHash(X, nbrs, 64, seed=21)))
        return run

    def with_hier(f):
        def run():
            f(hier)
        return run

    p = [
        ("philox block", lambda: rng_pins.test_philox_block_matches_numpy([5, 7], [1, 2, 3, 4])),
        ("projections seeded, pairs uncorrelated", rng_pins.test_projections_deterministic_and_seeded),
        ("projections standard normal", rng_pins.test_projections_are_standard_normal),
        ("projection layout", lambda: rng_pins.test_projection_layout_follows_the_counter_reading(3000, 128, 8, 16)),
        ("normal quantiles", const_pins.test_norm_ppf_textbook_values),
        ("eta", lambda: const_pins.test_eta_modes(16)),
        ("w_reg vs Lemma 5.4", lambda: const_pins.test_oracle_wreg_matches_lemma54_expectation(8, 128)),
        ("J_rel", const_pins.test_jrel_impact_of_L),
        ("Table 6", const_pins.test_table6_routing_test_comparison),
        ("codes L 8", lambda: codes_pins.test_codes_match_definitions(8, 128, 16)),
        ("codes L 1", lambda: codes_pins.test_codes_match_definitions(1, 64, 16)),
        ("equal block norms", codes_pins.test_equal_block_norms_give_zero_residual),
        ("degenerate edges", codes_pins.test_degenerate_edges),
        ("node tables", lambda: codes_pins.test_node_projection_table(8, 128)),
        ("BF16 = torch", prec_pins.test_bf16_equals_torch_rounding),
        ("E4M3 = torch", prec_pins.test_e4m3_equals_torch_rounding),
        ("E4M3 format facts", prec_pins.test_e4m3_format_facts_and_round_trip),
        ("rounding error bounds", prec_pins.test_rounding_error_bounds),
        ("compact extremes and error", lambda: compact_pins.test_extremes_and_error_bound(8)),
        ("compact half steps", lambda: compact_pins.test_half_steps_round_to_even_and_zero_nodes(8)),
        ("permutation example 1", lambda: perm_pins.test_worked_examples("ex1")),
        ("permutation example 2", lambda: perm_pins.test_worked_examples("ex2")),
        ("permutation rounds", lambda: perm_pins.test_greedy_round_invariants(96, 8, 1)),
        ("permuted index = permuted data", lambda: perm_pins.test_permutation_equals_permuted_data_and_queries(perm)),
        ("descent on a line", hier_pins.test_path_over_a_line_walks_to_the_nearest_point),
        ("descent ties", hier_pins.test_equal_neighbours_take_the_lower_id),
        ("complete layer", hier_pins.test_complete_layer_reaches_exact_nn),
        ("SimHash bits", lambda: sh_pins.test_bits_and_norms_match_definitions(64)),
        ("SimHash coverage and power", lambda: sh_pins.test_threshold_coverage_and_power(64, 0.1)),
        ("A, H, T unit scale", lambda: routing_pins.test_edge_statistics_match_definitions(0.2)),
        ("A, H, T sift scale", lambda: routing_pins.test_edge_statistics_match_definitions_sift_scale(0.2)),
        ("translated A = A_r", routing_pins.test_translated_A_is_paper_A_r),
        ("A rules and degenerate cases", routing_pins.test_a_rules_decide_by_distance_and_degenerate_cases_pass),
        ("knn brute force", search_pins.test_knn_f64_is_brute_force),
        ("efs = N exact", search_pins.test_full_ef_finds_exact_knn),
        ("ties with the bound", search_pins.test_ties_with_the_list_bound_are_not_inserted),
        ("generator graph = oracle graph", lambda: search_pins.test_generator_graph_equals_oracle_graph("tiny", 2000)),
        ("disabled test = plain", with_sift(search_pins.test_disabled_test_equals_plain_trajectory, 16)),
        ("results exact", with_sift(search_pins.test_results_sorted_and_exact)),
        ("PEOs saves distances", with_sift(search_pins.test_peos_saves_distances_at_similar_recall)),
        ("second implementation", with_sift(search_pins.test_lossy_visited_table_changes_nothing, 1, 256)),
        ("beam width", with_sift(search_pins.test_beam_width_follows_its_definition, 1, 2)),
        ("frame Q decides the comparison", with_glove(frameq_pins.test_frame_q_threshold_decides_the_distance_comparison)),
        ("frame Q statistic", with_glove(frameq_pins.test_frame_q_H_is_the_statistic_of_the_normalised_query)),
        ("frame Q decides the comparison, sift", with_sift_q(frameq_pins.test_frame_q_threshold_decides_the_distance_comparison)),
        ("frame Q statistic, sift", with_sift_q(frameq_pins.test_frame_q_H_is_the_statistic_of_the_normalised_query)),
        ("quantile table", with_glove(frameq_pins.test_quantile_table_is_slightly_conservative)),
        ("frame Q searches", with_glove(frameq_pins.test_frame_q_searches)),
        ("frame Q search = its test", frameq_pins.test_frame_q_search_follows_the_test_definition),
        ("SimHash search", with_sift_sh(sh_pins.test_search_follows_the_test_definition)),
        ("per-query entries", with_hier(hier_pins.test_per_query_entries)),
        ("re-rank of the full list = exact K-NN", with_glove(lambda g: prec_pins.test_rerank_with_full_list_is_exact_knn(g, 1))),
        ("lazy index reads the FP32 rows", with_glove(prec_pins.test_lazy_index_reads_fp32_rows_when_searching_stored_rows)),
        ("moments by Monte Carlo", routing_pins.test_estimator_moments_monte_carlo),
    ]
    return p


def _first_failure(path, pins):
    with oracle.using_library(path):
        for name, run in pins:
            try:
                run()
            except Exception as e:  # a pin that fails (assertion) or cannot finish
                return name, type(e).__name__
    return None


@pytest.fixture(scope="module")
def libraries(tmp_path_factory):
    """The unmodified copy and one library per planted mistake, compiled in parallel."""
    src = open(SRC).read()
    d = tmp_path_factory.mktemp("oracle_mutants")
    jobs = [("control", src)]
    for name, _, old, new in MUTATIONS:
        assert src.count(old) >= 1, f"{name}: the original text is not in the source"
        jobs.append((name, src.replace(old, new)))

    def compile_one(i_job):
        i, (name, text) = i_job
        c = os.path.join(d, f"m{i}.c")
        with open(c, "w") as f:
            f.write(text)
        so = os.path.join(d, f"libm{i}.so")
        oracle.compile_source(c, so)
        return name, so

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        return dict(ex.map(compile_one, enumerate(jobs)))


@pytest.fixture(scope="module")
def pins():
    return _pins(_small_sift(), _small_glove(), _small_simhash(), _small_hier(), _small_perm())


def test_unmodified_copy_passes_every_pin(libraries, pins):
    assert _first_failure(libraries["control"], pins) is None


@pytest.mark.parametrize("name", [m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(libraries, pins, name):
    caught = _first_failure(libraries[name], pins)
    assert caught is not None, f"no pin fails with the planted mistake: {name}"
