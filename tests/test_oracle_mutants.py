"""Planted-mistake check of the oracle's pins (CPU only).

Each case copies ``oracle/dawn_oracle.c``, plants one plausible mistake (a
wrong stamp, a dropped swap, the BOVM merge moved inside the vertex loop, a
transposed operand, a wrong bound in the certificate, ...), compiles the copy
into a temporary library and runs the pin suite against it through
``DAWN_ORACLE_SO``.  The pins must fail for every mutant.
"""
import os
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
SRC = ROOT / "oracle" / "dawn_oracle.c"

MUTANTS = {
    "sovm_wrong_stamp": ("beta[c] = 1;\n                    dist[c] = step;",
                         "beta[c] = 1;\n                    dist[c] = step + 1;"),
    "sovm_no_swap": ("(\"reset the vector by swap\") */\n        uint8_t* t = alpha;\n        alpha = beta;\n        beta = t;\n",
                     "(\"reset the vector by swap\") */\n        uint8_t* t = alpha;\n        (void)t;\n"),
    "sovm_restamps_source": ("if (dist[c] == -1) {\n                    beta[c] = 1;",
                             "if (dist[c] <= 0) {\n                    beta[c] = 1;"),
    "bovm_merge_inside_loop": ("beta[i] = 1;\n                    dist[i] = step;",
                               "beta[i] = 1; alpha[i] = 1;\n                    dist[i] = step;"),
    "bovm_transposed_operand": ("if (alpha[r] && r != i)", "if (alpha[i] && r != i)"),
    "bfs_wrong_increment": ("dist[c] = dist[i] + 1;", "dist[c] = dist[i] + 2;"),
    "floyd_wrong_arc_weight": ("if (c != i) d[(int64_t)i * n + c] = 1;", "if (c != i) d[(int64_t)i * n + c] = 2;"),
    "powers_off_by_one": ("d[(size_t)i * n + j] = k;", "d[(size_t)i * n + j] = k + 1;"),
    "cert_loose_bound": ("dist[v] > dist[u] + 1", "dist[v] > dist[u] + 2"),
    "cert_no_support_check": ("if (dist[v] == dist[u] + 1) supported[v] = 1;", "supported[v] = 1;"),
    "wcc_half_union": ("if (a < b) p[b] = a; else p[a] = b;", "if (a < b) p[b] = a;"),
    "msbfs_ecc_off_by_one": ("if (dist[v] > e) e = dist[v];", "if (dist[v] > e) e = dist[v] + 1;"),
    "msbfs_sum_counts": ("sum += dist[v];", "sum += 1;"),
    "harmonic_next_level": ("h += (double)count[d] / (double)d;", "h += (double)count[d] / (double)(d + 1);"),
    "closeness_counts_source": ("closeness[i] = r > 1 ? (double)(r - 1) / (double)sum : 0.0;",
                                "closeness[i] = r > 1 ? (double)r / (double)sum : 0.0;"),
    "radius_counts_isolated": ("if (r > 1 && (small < 0 || e < small)) small = e;", "if (small < 0 || e < small) small = e;"),
    "parents_largest_id": ("(parent[v] < 0 || u < parent[v])) parent[v] = u;", "(parent[v] < 0 || u > parent[v])) parent[v] = u;"),
    "parents_same_level_too": ("if (dist[v] == dist[u] + 1 && (parent[v] < 0", "if (dist[v] >= dist[u] && dist[v] > 0 && (parent[v] < 0"),
    "minplus_ignores_weight": ("const int64_t nd = dprev[i] + (int64_t)w[j];", "const int64_t nd = dprev[i] + 1;"),
    "minplus_current_values": ("const int64_t nd = dprev[i] + (int64_t)w[j];", "const int64_t nd = d[i] + (int64_t)w[j];"),
    "minplus_nonstrict": ("if (nd < d[c]) {\n                    d[c] = nd;", "if (nd <= d[c]) {\n                    d[c] = nd;"),
    "dijkstra_drops_key": ("const int64_t nd = it.key + (int64_t)w[j];", "const int64_t nd = (int64_t)w[j];"),
    "wcert_no_tight_search": ("if (dist[v] >= 0 && !seen[v]) { *bad = v; ok = 0; }",
                              "if (0 && dist[v] >= 0 && !seen[v]) { *bad = v; ok = 0; }"),
    "wcert_loose_bound": ("if (dist[v] < 0 || dist[v] > dist[u] + (int64_t)w[j]) { *bad = v; return 0; }",
                          "if (dist[v] < 0 || dist[v] > dist[u] + (int64_t)w[j] + 1) { *bad = v; return 0; }"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    text = SRC.read_text()
    assert text.count(old) == 1, f"mutation site for {name} not unique"
    src = tmp_path / "mutant.c"
    src.write_text(text.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(src)], check=True)
    env = dict(os.environ, DAWN_ORACLE_SO=str(so))
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                          str(ROOT / "tests" / "test_oracle_pins.py")],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode != 0, f"pins did not catch mutant {name}:\n{res.stdout[-2000:]}"
