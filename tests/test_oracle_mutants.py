"""Planted mistakes in the oracle must be caught by its pins.

Each mutant is one plausible slip (a wrong comparison, a dropped update, a
wrong index) applied to a temporary copy of ``oracle/oracle.c``. The copy is
compiled and loaded in a subprocess, which runs a small pin battery: the
brute-force definition on random graphs, closed forms and the paper's G1,
for every rendition (BZ, Alg. 2, 3, 4, 6, NbrCore, CntCore), plus the
hand-counted step structure of GPP and the round counts of the Index2core
renditions.
The battery must pass on the unmodified source and fail on every mutant.
"""
import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    # Batagelj-Zaversnik
    "bz-ge": ("if (deg[u] > deg[v]) {", "if (deg[u] >= deg[v]) {"),
    "bz-no-bin-move": ("bin[du]++;\n                deg[u]--;", "deg[u]--;"),
    "bz-no-swap": ("if (u != w) {", "if (0) {"),
    "bz-no-bin-shift": ("for (int32_t d = md; d >= 1; --d) bin[d] = bin[d - 1];\n    bin[0] = 0;", ""),
    "bz-wrong-slot": ("int64_t pw = bin[du];", "int64_t pw = pos[u];"),
    # HINDEX (Alg. 2) and the checker
    "hindex-strict": ("if (s >= h) break;\n    }\n    return h;", "if (s > h) break;\n    }\n    return h;"),
    "hindex-off-by-one": ("int32_t x = val[ci[e]];", "int32_t x = val[ci[e]] > 0 ? val[ci[e]] - 1 : 0;"),
    "check-certificate": ("if (ge < c) out[1]++;", "if (ge + 1 < c) out[1]++;"),
    # PeelOne (Alg. 4)
    "peel-ge": ("if (core[u] > k) {\n                        core[u] -= 1;",
                "if (core[u] >= k) {\n                        core[u] -= 1;"),
    "peel-no-dynamic-frontier": ("if (core[u] == k) q[qtail++] = u;", ""),
    # HistoCore (Alg. 6)
    "histo-sum-strict": ("if (sum >= k) break;", "if (sum > k) break;"),
    "histo-no-cnt-store": ("histo[rp[v] + k - 1] = (int32_t)sum;", ""),
    "histo-late-push": ("if (x >= K && old == K) {", "if (x >= K && old == K - 1) {"),
    "histo-no-increment": ("histo[rp[u] + y - 1] += 1;", ""),
    "histo-init-slot": ("histo[rp[v] + (du < dv ? du : dv) - 1] += 1;",
                        "histo[rp[v] + dv - 1] += 1;"),
    # GPP (Alg. 3)
    "gpp-strict-frontier": ("if (!rem[v] && deg[v] <= k) front[nf++] = (int32_t)v;",
                            "if (!rem[v] && deg[v] < k) front[nf++] = (int32_t)v;"),
    "gpp-no-rem-guard": ("if (!rem[ci[e]]) { deg[ci[e]]--; st[2]++; }", "{ deg[ci[e]]--; st[2]++; }"),
    "gpp-k-skip": ("if (nf == 0) { k++; continue; }", "if (nf == 0) { k += 2; continue; }"),
    # NbrCore / CntCore
    "i2c-cnt-strict": ("c += (core[ci[e]] >= core[v]);", "c += (core[ci[e]] > core[v]);"),
    "i2c-in-place": ("chg[nchg] = v;\n                newv[nchg++] = h;",
                     "chg[nchg] = v;\n                newv[nchg++] = h;\n                core[v] = h;"),
    "i2c-no-neighbours": ("if (!mark[ci[e]]) { mark[ci[e]] = 1; nxt[nn2++] = ci[e]; }",
                          "if (!mark[v]) { mark[v] = 1; nxt[nn2++] = v; }"),
}

BATTERY = textwrap.dedent(r"""
    import sys, itertools
    import numpy as np
    sys.path[:0] = [{root!r}, {tests!r}]
    import oracle
    oracle._SRC, oracle._LIB, oracle._lib = {src!r}, {so!r}, None
    import graphgen as gg
    from conftest import load_g1

    fails = []

    def run(tag, n, edges, want):
        rp, ci = gg.from_edge_list(edges, n).numpy()
        got = {{
            "bz": oracle.bz_coreness(rp, ci),
            "jacobi": oracle.hindex_jacobi(rp, ci)[0],
            "peel": oracle.peelone(rp, ci)[0],
        }}
        h, st = oracle.histocore(rp, ci, check=True)
        got["histo"] = h
        got["gpp"], gst = oracle.gpp(rp, ci)
        jr = oracle.hindex_jacobi(rp, ci)[1]
        for nm, fn in (("nbr", oracle.nbrcore), ("cnt", oracle.cntcore)):
            got[nm], ist = fn(rp, ci)
            if ist["rounds"] != jr or ist["frontier"] != st["frontier"] or ist["violations"]:
                fails.append((tag, nm + "-rounds"))
        if gst["scans"] != gst["steps"] + max(want + [0]):
            fails.append((tag, "gpp-scans"))
        for k, v in got.items():
            if list(v) != list(want):
                fails.append((tag, k))
        if st["violations"]:
            fails.append((tag, "histo-invariant"))
        w = np.array(want, dtype=np.int32)
        if any(oracle.check(rp, ci, w).values()):
            fails.append((tag, "check-rejects-truth"))
        for v in range(n):
            if want[v] > 0:
                bad = w.copy(); bad[v] += 1
                if not any(oracle.check(rp, ci, bad).values()):
                    fails.append((tag, "check-accepts-raised"))
                break

    # each component of the checker on fixed vectors, counted by hand:
    # K4 with (3,3,3,2): v0..v2 see two neighbours >= 3 (certificate fails
    # for 3 vertices); HINDEX is 2 for v0..v2 and 3 for v3 (4 fixpoint misses).
    k4 = gg.complete_graph(4).numpy()
    if oracle.check(*k4, np.array([3, 3, 3, 2], np.int32)) != {{"range": 0, "certificate": 3, "fixpoint": 4}}:
        fails.append(("K4", "check-components"))
    if oracle.check(*k4, np.zeros(4, np.int32)) != {{"range": 0, "certificate": 0, "fixpoint": 0}}:
        fails.append(("K4", "check-zero"))
    p3 = gg.path_graph(3).numpy()
    if oracle.check(*p3, np.array([1, 3, 1], np.int32)) != {{"range": 1, "certificate": 0, "fixpoint": 0}}:
        fails.append(("P3", "check-range"))

    # GPP on paths, counted by hand: ceil(n/2) steps, n - 2 (even n) or
    # n - 1 (odd n) decrements
    for pn in (4, 5, 8):
        _, gst = oracle.gpp(*gg.path_graph(pn).numpy())
        if (gst["steps"], gst["decrements"]) != ((pn + 1) // 2, pn - 2 if pn % 2 == 0 else pn - 1):
            fails.append((f"P{{pn}}", "gpp-steps"))

    n, edges, want = load_g1()
    run("G1", n, edges, want)
    for name, g, k in [("K6", gg.complete_graph(6), 5), ("C7", gg.cycle_graph(7), 2),
                       ("P5", gg.path_graph(5), 1), ("grid4x5", gg.grid_graph(4, 5), 2),
                       ("Q4", gg.hypercube(4), 4), ("K3,5", gg.complete_bipartite(3, 5), 3)]:
        rp, ci = g.numpy()
        nn, ee = oracle.csr_to_edges(rp, ci)
        run(name, nn, ee, [k] * nn)
    rng = np.random.default_rng(7)
    for t in range(40):
        nn = int(rng.integers(6, 31))
        p = [0.1, 0.2, 0.35, 0.5][t % 4]
        ee = [(u, v) for u in range(nn) for v in range(u + 1, nn) if rng.random() < p]
        run(f"rand{{t}}", nn, ee, oracle.brute_force_coreness(nn, ee))
    print("FAILS", len(fails), fails[:5])
    sys.exit(1 if fails else 0)
""")


def _run_battery(tmp_path, source: str) -> subprocess.CompletedProcess:
    c = tmp_path / "oracle.c"
    c.write_text(source)
    so = tmp_path / "liboracle.so"
    script = BATTERY.format(root=ROOT, tests=os.path.join(ROOT, "tests"), src=str(c), so=str(so))
    return subprocess.run([sys.executable, "-c", script], capture_output=True, text=True,
                          timeout=300)


def test_battery_accepts_unmodified_oracle(tmp_path):
    with open(SRC) as f:
        src = f.read()
    r = _run_battery(tmp_path, src)
    assert r.returncode == 0, r.stdout + r.stderr


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_battery_rejects_mutant(tmp_path, name):
    with open(SRC) as f:
        src = f.read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site of {name} not unique"
    r = _run_battery(tmp_path, src.replace(old, new))
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout}{r.stderr}"
