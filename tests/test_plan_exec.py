"""CPU check of whole transform plans: every launch of a TFT / ITFT plan, run job by job on
Python values, against the oracle.

zx_transform_jobs returns the launches tft_ex / itft_ex make (in stream order), each job's
descriptor and the job images. A launch's jobs run concurrently on the GPU, so here each
launch reads the buffer as the previous launch left it and its stores land together. Besides
the values, the plans must be safe to run as launches of independent CTAs:

  * every cell a job reads or writes lies in [0, L);
  * within one launch, no two jobs store the same cell and no job reads a cell another job
    stores;
  * a job that stores the kernel's internal form (pad bit 8) only stores cells that a later
    launch stores again, so every output leaves in canonical form.

The arithmetic is Python integers, so this checks the planner's passes, strides, weights,
scaling and bookkeeping (Algorithms 1 and 2 split into passes, Secs. 3-4), not the limb
arithmetic of the kernel.
"""
import random

import pytest

from jobsim import Fermat, run_image

JOB_RAW_STORE = 1 << 8


@pytest.fixture(scope="module")
def tg():
    import paper_0810_3203_gb300 as m
    m.build.build()
    m.load(build_if_missing=False)
    return m


def job_cells(jd, count):
    return [jd["cell0"] + m * jd["mstride"] for m in range(count)]


def check_plan_safety(plan, L, outputs):
    """The launch-level properties of the module docstring; returns nothing, asserts."""
    launches = plan["launches"]
    stored_by = []  # per launch: the set of cells it stores
    for k, launch in enumerate(launches):
        stores, loads = {}, {}
        for t, jd in enumerate(launch["jobs"]):
            for c in job_cells(jd, max(jd["nload"], jd["nstore"])):
                assert 0 <= c < L, (k, t, c)
            for c in job_cells(jd, jd["nstore"]):
                assert c not in stores, f"launch {k}: cell {c} stored by jobs {stores[c]} and {t}"
                stores[c] = t
            for c in job_cells(jd, jd["nload"]):
                loads.setdefault(c, set()).add(t)
        for c, t in stores.items():
            assert loads.get(c, {t}) <= {t}, f"launch {k}: cell {c} stored by job {t}, read by {loads[c]}"
        stored_by.append(set(stores))
    later = set()
    for k in range(len(launches) - 1, -1, -1):
        for t, jd in enumerate(launches[k]["jobs"]):
            if jd["pad"] & JOB_RAW_STORE:
                cells = set(job_cells(jd, jd["nstore"]))
                assert cells <= later, f"launch {k} job {t}: internal form stored but never rewritten"
        later |= stored_by[k]
    assert set(outputs) <= later, "an output cell is never stored"


def run_plan(plan, N, vals, L, mode=0):
    """The buffer after every launch of the plan, from inputs `vals` (zeros beyond them)."""
    R = Fermat(N, mode)
    x = list(vals) + [0] * (L - len(vals))
    for launch in plan["launches"]:
        out = {}
        for jd in launch["jobs"]:
            ls = (jd["pad"] & 0xFF) or launch["ls"]
            cells = job_cells(jd, max(jd["nload"], jd["nstore"]))
            inputs = [x[c] for c in cells[:jd["nload"]]]
            got = run_image(plan["images"][jd["image"]], ls, N, jd["e"], inputs, jd["nload"], jd["nstore"],
                            jd["nscale"], jd["escale"], ring=R)
            for m, v in got.items():
                out[cells[m]] = v
        for c, v in out.items():
            x[c] = v
    return x


def oracle_transform(orc, kind, vals, l, z, n, f, e, N, mode):
    x = orc.cells_from_ints(vals, N, count=1 << l)
    if kind == 0:
        (orc.sqrt2_tft if mode == 2 else orc.tft)(x, l, z, n, e, N)
        return orc.cells_to_ints(x, N, n)
    (orc.sqrt2_itft if mode == 2 else orc.itft)(x, l, z, n, f, e, N)
    return orc.cells_to_ints(x, N, n + f)


def check_case(tg, orc, kind, l, z, n, f, e, N, scale=0, mode=0, seed=0):
    L = 1 << l
    p = (1 << N) + 1
    rng = random.Random(seed)
    vals = [rng.randrange(p) for _ in range(z)]
    # structured cells too: 0, -1 = 2^N and 1
    for i, v in zip(range(0, z, max(1, z // 3)), (0, p - 1, 1)):
        vals[i] = v
    plan = tg.transform_jobs(kind, l, z, n, N, f=f, e=e, scale=scale, mode=mode)
    outs = n if kind == 0 else n + f
    check_plan_safety(plan, L, range(outs))
    got = run_plan(plan, N, vals, L, mode)[:outs]
    want = oracle_transform(orc, kind, vals, l, z, n, f, e, N, mode)
    if kind == 1 and scale:
        inv = pow(2, -l, p)
        want = [v * inv % p for v in want[:n]] + want[n:]
    assert got == want, (kind, l, z, n, f, e, N, scale, mode)
    return plan


# (kind, l, z, n, f, e, N, scale): single launches, two-pass plans (more than 64 cells) and
# ragged lengths on both sides of the row boundaries
DEFAULT_CASES = [
    (0, 6, 40, 37, 0, 5, 256, 0),
    (1, 6, 40, 37, 1, 5, 256, 0),
    (0, 9, 300, 300, 0, 0, 1024, 0),
    (1, 9, 300, 300, 0, 0, 1024, 1),
    (0, 10, 1024, 1024, 0, 17, 1024, 0),
    (1, 10, 1024, 1000, 1, 17, 1024, 0),
    (0, 11, 1500, 1999, 0, 3, 1024, 0),
    (1, 11, 1999, 1500, 1, 3, 1024, 1),
    (1, 11, 1025, 1025, 0, 0, 1024, 1),
    (0, 12, 2049, 2049, 0, 1, 2048, 0),
]


@pytest.mark.parametrize("case", DEFAULT_CASES)
def test_default_plans_match_the_oracle(tg, orc, case):
    kind, l, z, n, f, e, N, scale = case
    check_case(tg, orc, kind, l, z, n, f, e, N, scale, seed=l * 7 + kind)


# pinned launch configurations: 8-cell single-CTA jobs with 64-cell jobs on 8-CTA clusters,
# 4-cell jobs with 16-cell jobs on 4-CTA clusters, the ceil(l/2) top split
PINNED = [
    dict(ls_max=3, ls_c=3, max_warps=8, split=0),
    dict(ls_max=2, ls_c=2, max_warps=16, split=1),
    dict(ls_max=4, ls_c=2, max_warps=8, split=1),
    # the fewest-pass split with clusters of at most 4 or 2 CTAs
    dict(ls_max=3, ls_c=3, max_warps=8, split=2, max_cluster_log2=2),
    dict(ls_max=3, ls_c=4, max_warps=16, split=2, max_cluster_log2=1),
]


@pytest.mark.parametrize("cfg", PINNED, ids=lambda c: f"ls{c['ls_max']}c{c['ls_c']}s{c['split']}m{c.get('max_cluster_log2', 4)}")
def test_pinned_configurations_match_the_oracle(tg, orc, cfg):
    N = 2048
    before = tg.config_get(N)
    tg.config_set(N, cfg)
    try:
        rng = random.Random(cfg["ls_max"] * 31 + cfg["split"])
        passes = set()
        for kind, l, z, n, f in ((0, 12, 4096, 4096, 0), (1, 12, 4096, 4096, 0), (0, 11, 1333, 1700, 0),
                                 (1, 11, 1700, 1333, 1), (1, 12, 3001, 2999, 1), (0, 9, 200, 511, 0)):
            e = rng.randrange(2 * N)
            plan = check_case(tg, orc, kind, l, z, n, f, e, N, scale=kind, seed=l + 3 * kind + n)
            passes.add(plan["passes"])
            assert any(L["lc"] > 0 for L in plan["launches"]) or cfg["ls_c"] < 3 or l < 12
            assert all(L["lc"] <= cfg.get("max_cluster_log2", 4) for L in plan["launches"])
        assert max(passes) >= 3  # these configurations split the transforms into several passes
    finally:
        tg.config_set(N, before)


@pytest.mark.parametrize("kind,l,z,n,f", [(0, 10, 700, 1024, 0), (1, 10, 1024, 900, 1), (0, 11, 2048, 1500, 0)])
def test_sqrt2_plans_match_the_oracle(tg, orc, kind, l, z, n, f):
    """omega = sqrt2 (L | 4N): rotation amounts mod 4N, the odd powers of sqrt2 included."""
    N = 512
    check_case(tg, orc, kind, l, z, n, f, 11, N, scale=kind, mode=2, seed=l + kind)


def test_the_benchmark_plan_is_safe(tg):
    """The l = 16, N = 32768 plans of the benchmark's n (too large to run in Python): every
    launch-level property, and the internal form on all but the last pass."""
    L = 1 << 16
    for n in (32769, 40000, 45000, 52000, 65536):
        for kind in (0, 1):
            plan = tg.transform_jobs(kind, 16, n, n, 32768, scale=kind)
            check_plan_safety(plan, L, range(n))
            raw = [any(jd["pad"] & JOB_RAW_STORE for jd in launch["jobs"]) for launch in plan["launches"]]
            assert not raw[-1] and (kind == 1 or all(raw[:-1])), (kind, n, raw)


def test_the_profiled_plan_shape(tg):
    """The TFT at n = 40000, l = 16, N = 32768 under its default configuration is the plan the
    ncu summaries describe: four passes of 16-cell single-CTA jobs, 4096, 2560, 2512 and 2500
    jobs (one CTA each), all but the last storing the internal form where they may. A job
    stores canonical cells when one of its cells is never stored again:

      * pass 1: top column u's 256-cell TFT (height 157) splits 16 x 16, and its inner column c
        stores inner rows 0..9 (rows 16 r + c). Pass 2 stores rows below 157 only, so inner
        columns 13, 14, 15 of every top column stay canonical: 3 x 256 = 768 jobs.
      * pass 2: inner row 9 of top column u stores row 156. The last row's TFT outputs only
        columns below n2 = 64, so the 256 - 64 = 192 columns from 64 on stay canonical."""
    plan = tg.transform_jobs(0, 16, 40000, 40000, 32768)
    assert plan["passes"] == 4
    assert [len(L["jobs"]) for L in plan["launches"]] == [4096, 2560, 2512, 2500]
    assert all(L["lc"] == 0 and L["ls"] == 4 for L in plan["launches"])
    canonical = [sum(not jd["pad"] & JOB_RAW_STORE for jd in L["jobs"]) for L in plan["launches"]]
    assert canonical == [768, 192, 0, 2500], canonical


def test_plan_safety_sweep(tg):
    """The launch-level rules (no execution) over ring sizes, lengths and both transforms:
    every cell in bounds, no cell written by two CTAs of one launch or read by one while
    another writes it, internal-form stores always rewritten. Includes the padded lengths the
    products' zero-padded ITFT uses at the benchmark's size."""
    rng = random.Random(2024)
    cases = []
    for N, lmax in ((64, 7), (1024, 11), (4096, 13), (32768, 16)):
        for l in range(1, lmax + 1):
            L = 1 << l
            for _ in range(3 if l < lmax else 6):
                n = rng.randint(1, L)
                cases.append((0, l, rng.randint(1, L), n, 0, N))
                f = rng.randint(0, 1) if n < L else 0
                cases.append((1, l, rng.randint(n, L), n, f, N))
    for n in (33024, 40192, 45056, 52224):
        cases.append((1, 16, n, n, 0, 32768))
        cases.append((0, 16, n, n, 0, 32768))
    cases = [c + (0,) for c in cases]
    # omega = sqrt2: L | 4N, one level more per ring
    for N, lmax in ((64, 8), (1024, 12), (8192, 15)):
        for l in range(lmax - 3, lmax + 1):
            L = 1 << l
            n = rng.randint(1, L)
            cases.append((0, l, rng.randint(1, L), n, 0, N, 2))
            cases.append((1, l, rng.randint(n, L), n, 1 if n < L else 0, N, 2))
    for kind, l, z, n, f, N, mode in cases:
        plan = tg.transform_jobs(kind, l, z, n, N, f=f, e=rng.randrange(2 * N), scale=kind, mode=mode)
        check_plan_safety(plan, 1 << l, range(n if kind == 0 else n + f))


def test_tft_plans_come_levelled(tg):
    """The planner takes an Algorithm 1 plan's passes as its dependency levels without
    relevelling them: a sub-transform reads all of its inputs in its first pass, so each pass
    reads a cell the pass before it stored. Checked here from the outside on plans of single-CTA
    jobs (one launch per pass), and no launch may be empty."""
    rng = random.Random(77)
    checked = 0
    for N, lmax in ((64, 7), (1024, 11), (4096, 12), (32768, 13)):
        for l in range(2, lmax + 1):
            L = 1 << l
            for _ in range(4 if l < 10 else 2):
                z, n = rng.randint(1, L), rng.randint(1, L)
                plan = tg.transform_jobs(0, l, z, n, N)
                launches = plan["launches"]
                if any(launch["lc"] for launch in launches):
                    continue
                assert len(launches) == plan["passes"], (l, z, n, N)
                assert all(launch["jobs"] for launch in launches)
                for prev, cur in zip(launches, launches[1:]):
                    stored = {jd["cell0"] + m * jd["mstride"] for jd in prev["jobs"] for m in range(jd["nstore"])}
                    read = {jd["cell0"] + m * jd["mstride"] for jd in cur["jobs"] for m in range(jd["nload"])}
                    assert stored & read, (l, z, n, N)
                checked += 1
    assert checked > 60


def test_snake_order_only_in_plans_larger_than_half_of_l2(tg):
    """Plans whose cells exceed 64 MB take every other launch's jobs in reverse order, so that a
    pass starts on the cells the pass before it stored last; smaller plans (they fit in L2) keep
    the sorted order. The l = 16 TFT at n = 40000, N = 32768 spans 40960 cells of 4104 bytes."""
    big = tg.transform_jobs(0, 16, 40000, 40000, 32768)["launches"]
    firsts = [launch["jobs"][0]["cell0"] for launch in big]
    lasts = [launch["jobs"][-1]["cell0"] for launch in big]
    assert [f < l for f, l in zip(firsts, lasts)] == [True, False, True, False], (firsts, lasts)
    small = tg.transform_jobs(0, 13, 6000, 6000, 8192)["launches"]
    assert all(launch["jobs"][0]["cell0"] <= launch["jobs"][-1]["cell0"] for launch in small)


def test_concurrent_planning_matches_sequential_planning(tg):
    """The planner keeps its job lists and per-cell scratch in per-thread buffers that outlive a
    plan. Plans made on four threads at once (the foreign calls release the interpreter lock)
    must equal the same plans made one after another, in every job field and image."""
    import threading

    rng = random.Random(5)
    cases = []
    for N, lmax in ((1024, 11), (4096, 12), (32768, 13)):
        for _ in range(6):
            l = rng.randint(4, lmax)
            L = 1 << l
            n = rng.randint(1, L)
            if rng.random() < 0.5:
                cases.append((0, l, rng.randint(1, L), n, 0, N))
            else:
                cases.append((1, l, rng.randint(n, L), n, 1 if n < L and rng.random() < 0.5 else 0, N))

    def key(plan):
        return (plan["passes"], [(launch["ls"], launch["lc"], launch["warps"], launch["program_words"],
                                  [tuple(sorted(jd.items())) for jd in launch["jobs"]]) for launch in plan["launches"]],
                [img.tobytes() for img in plan["images"]])

    expected = [key(tg.transform_jobs(kind, l, z, n, N, f=f)) for kind, l, z, n, f, N in cases]
    results = [[None] * len(cases) for _ in range(4)]
    errors = []

    def worker(t):
        try:
            for _ in range(3):
                for i in rng_orders[t]:
                    kind, l, z, n, f, N = cases[i]
                    got = key(tg.transform_jobs(kind, l, z, n, N, f=f))
                    if results[t][i] is None or got != expected[i]:
                        results[t][i] = got
        except Exception as exc:  # reported below
            errors.append(exc)

    rng_orders = []
    for t in range(4):
        order = list(range(len(cases)))
        random.Random(t).shuffle(order)
        rng_orders.append(order)
    threads = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    for t in range(4):
        for i in range(len(cases)):
            assert results[t][i] == expected[i], (t, cases[i])


def test_the_fewest_pass_plan_at_the_benchmark_size(tg):
    """split 2 with clusters of at most 4 CTAs and 16 cells per cluster CTA: the l = 16 TFT at
    N = 32768 takes three global-memory passes (64-cell column jobs on 4-CTA clusters, then rows
    of 32 cells) against four for the paper's split, the exact ITFT three to eight (the partial
    rows of Algorithm 2 add steps) against twelve; the launch rules hold for both."""
    N = 32768
    before = tg.config_get(N)
    tg.config_set(N, dict(before, ls_c=4, split=2, max_cluster_log2=2))
    try:
        for n in (32769, 40000, 45000, 65536):
            tft = tg.transform_jobs(0, 16, n, n, N)
            itft = tg.transform_jobs(1, 16, n, n, N, scale=1)
            assert tft["passes"] == 3 and len(tft["launches"]) == 3, n
            assert tft["launches"][0]["ls"] == 6 and tft["launches"][0]["lc"] == 2
            assert itft["passes"] <= 8 and len(itft["launches"]) <= 8, n
            check_plan_safety(tft, 1 << 16, range(n))
            check_plan_safety(itft, 1 << 16, range(n))
    finally:
        tg.config_set(N, before)
