"""Planted mistakes: each is a plausible slip in the oracle (a dropped term, a
flipped sign or comparison, a wrong operand).  A copy of gp_oracle.c with the
slip applied is compiled on the CPU and the pin suite is run against it in a
subprocess; every slip must make at least one pin fail."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gp_oracle.c")

MUTATIONS = {
    "makespan_drops_transfer": ("const int64_t t = fin[v] + (part[u] != part[v] ? w[e] : 0);",
                                "const int64_t t = fin[v];"),
    "makespan_wrong_side_cost": ("fin[v] = start[v] + (part[v] ? cG[v] : cC[v]);",
                                 "fin[v] = start[v] + (part[v] ? cC[v] : cG[v]);"),
    "eq1_wrong_numerator": ("((i128)SC * (i128)SG) / den", "((i128)SC * (i128)SC) / den"),
    "bounds_drop_tolerance": ("const i128 scale = (i128)1000000 + ppm;", "const i128 scale = (i128)1000000;"),
    "symmetrize_one_direction": ("      raw[fill[v]].w = w[e];", "      raw[fill[v]].w = 0;"),
    "match_light_edges": ("if (x->W != y->W) return x->W > y->W;", "if (x->W != y->W) return x->W < y->W;"),
    "match_hash_reversed": ("if (x->h != y->h) return x->h > y->h;", "if (x->h != y->h) return x->h < y->h;"),
    "match_not_mutual": ("if (u >= 0 && pick[u] == (int32_t)v) mate[v] = u;", "if (u >= 0) mate[v] = u;"),
    "match_ignores_cpu_cap": ("if (vC[v] + vC[u] > capC || vG[v] + vG[u] > capG) continue;",
                              "if (vG[v] + vG[u] > capG) continue;"),
    "twohop_ignores_caps": ("if (pending >= 0 && vC[pending] + vC[v] <= capC && vG[pending] + vG[v] <= capG &&",
                            "if (pending >= 0 &&"),
    "contract_no_weight_sum": ("      cvC[c] += vC[x];", "      cvC[c] = vC[x];"),
    "contract_keeps_self": ("        if (t == c) continue;\n", ""),
    "gain_sign_flipped": ("    gain[v] = ext - in;", "    gain[v] = in - ext;"),
    "refine_ignores_bound": ("        if (acc + c > Bd - Ld) break;", "        if (acc > Bd - Ld) break;"),
    "refine_wrong_order": ("if (x->gain != y->gain) return x->gain > y->gain ? -1 : 1;",
                           "if (x->gain != y->gain) return x->gain < y->gain ? -1 : 1;"),
    "balance_longest_prefix": ("        k = i;\n        break;", "        k = i;"),
    "gggp_gain_flipped": ("const int64_t g = 2 * toC[v] - wsum[v];", "const int64_t g = wsum[v] - 2 * toC[v];"),
    "gggp_ignores_adjacency": ("const int a = adjC[v] > 0;", "const int a = 0;"),
    "gggp_worst_trial": ("(feas == best_feas && cut < best_cut)", "(feas == best_feas && cut > best_cut)"),
    "cut_counts_internal": ("if (part[u] != part[cols[e]]) c += w[e];", "if (part[u] == part[cols[e]]) c += w[e];"),
    "stall_rule_inverted": ("if (nc * OG_STALL_DEN > f->n * OG_STALL_NUM) {", "if (nc * OG_STALL_DEN < f->n * OG_STALL_NUM) {"),
    "fixed_match_ignores_pins": ("        if (!og_compatible(fix, v, u)) continue;\n", ""),
    "fixed_twohop_ignores_pins": (" &&\n          og_compatible(fix, pending, v)) {", ") {"),
    "fixed_coarse_pin_lost": ("if (f->fix[v] > c->fix[f->cmap[v]])", "if (f->fix[v] < c->fix[f->cmap[v]])"),
    "fixed_grow_moves_pins": ("if (side[v] != 1 || (fix && fix[v] >= 0) || LC + vC[v] > BC) continue;",
                              "if (side[v] != 1 || LC + vC[v] > BC) continue;"),
    "fixed_grow_start_pinned": ("const int start_free = !fix || fix[start] < 0;", "const int start_free = 1;"),
    "fixed_refine_moves_pins": ("if (part[v] == src && gain[v] > 0 && !(fix && fix[v] >= 0)) {",
                                "if (part[v] == src && gain[v] > 0) {"),
    "fixed_balance_moves_pins": ("if (part[v] == s && !(fix && fix[v] >= 0)) {", "if (part[v] == s) {"),
    "fixed_grow_region_empty": ("    side[v] = (fix && fix[v] == 0) ? 0 : 1;\n    toC[v] = 0;",
                                "    side[v] = 1;\n    toC[v] = 0;"),
    "listsched_ignores_transfer": ("const int64_t arrive = fin[u] + (part[u] != part[v] ? w[e] : 0);",
                                   "const int64_t arrive = fin[u];"),
    "listsched_starts_before_data": ("while (idle[s] > 0 && wlen[s] > 0 && wait[s][0].t <= t) {",
                                     "while (idle[s] > 0 && wlen[s] > 0) {"),
    "listsched_ties_larger_id_first": ("return a->t < b->t || (a->t == b->t && a->v < b->v);",
                                       "return a->t < b->t || (a->t == b->t && a->v > b->v);"),
    "listsched_order_by_id_only": ("return a->t < b->t || (a->t == b->t && a->v < b->v);", "return a->v < b->v;"),
    "listsched_worker_never_freed": ("      idle[part[u]]++;\n", ""),
    "listsched_wrong_side_cost": ("fin[v] = t + (part[v] ? cG[v] : cC[v]);", "fin[v] = t + (part[v] ? cC[v] : cG[v]);"),
    "vcycle_refine_keeps_pins": ("                      restrict_only ? NULL : lv[l].fix, BC, BG, pc, &rs) != OG_OK)",
                                 "                      lv[l].fix, BC, BG, pc, &rs) != OG_OK)"),
    "vcycle_coarsest_all_gpu": ("for (int64_t x = 0; x < lv[L].n; x++) pc[x] = (uint8_t)lv[L].fix[x];",
                                "for (int64_t x = 0; x < lv[L].n; x++) pc[x] = 1;"),
    "kway_group_time_summed": ("  return (int64_t)(((__int128)x * (__int128)y) / (__int128)(x + y));", "  return x + y;"),
    "kway_mid_rounded_down": ("const int mid = lo + (hi - lo + 1) / 2;", "const int mid = lo + (hi - lo) / 2;"),
    "kway_sides_swapped": ("rc = og_bisect(sn, soff, scols, sw, n_all, costs, sorig, side ? mid : lo, side ? hi : mid, tol, seed, cls,",
                           "rc = og_bisect(sn, soff, scols, sw, n_all, costs, sorig, side ? lo : mid, side ? mid : hi, tol, seed, cls,"),
    "kway_subgraph_loses_edges": ("        if (part[cols[e]] == side) {", "        if (0) {"),
    "no_twohop_in_pipeline": ("        og_match_twohop_fix(f->n, f->off, f->adj, f->W, f->vC, f->vG, f->fix, capC, capG, seed,\n"
                              "                            mate) != OG_OK) {", "        0) {"),
}


def _run(name, old, new, tmp):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation %s does not apply exactly once" % name
    d = os.path.join(tmp, name)
    os.makedirs(d)
    shutil.copy(os.path.join(ROOT, "oracle", "gp_oracle.h"), d)
    with open(os.path.join(d, "gp_oracle.c"), "w") as f:
        f.write(src.replace(old, new))
    so = os.path.join(d, "lib.so")
    subprocess.check_call(["gcc", "-std=gnu11", "-O1", "-w", "-shared", "-fPIC", "-o", so,
                           os.path.join(d, "gp_oracle.c"), "-lm"])
    env = dict(os.environ, GP_ORACLE_LIB=so, PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-400:]


def test_every_planted_mistake_fails_a_pin():
    with tempfile.TemporaryDirectory() as tmp:
        with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
            futs = {k: ex.submit(_run, k, a, b, tmp) for k, (a, b) in MUTATIONS.items()}
            survivors = {}
            for k, f in futs.items():
                rc, out = f.result()
                if rc == 0:
                    survivors[k] = out
    assert not survivors, "planted mistakes not caught: %s" % sorted(survivors)
