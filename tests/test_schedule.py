"""CPU check of the persistent form of transform plans (zx_transform_schedule).

A plan whose jobs all run on single CTAs is enqueued as one launch: its CTAs claim the jobs in
a fixed order and a claimed job waits until the jobs listed for it have finished. On the GPU,
any job whose listed jobs are done may run at any moment, so the lists must order every pair
of jobs that touch a common cell when one of them stores it. Here the jobs run one at a time on
Python integers, in random orders that respect the lists (and in the claim order itself), and
the result must equal the oracle's TFT / ITFT (Algorithms 1 and 2, Secs. 3-4) every time. For
the benchmark's l = 16 plans, too large to execute, the lists are checked against the cells the
jobs read and store.
"""
import random

import pytest

from jobsim import Fermat, run_image
from test_plan_exec import job_cells, oracle_transform


@pytest.fixture(scope="module")
def tg():
    import paper_0810_3203_gb300 as m
    m.build.build()
    m.load(build_if_missing=False)
    # the persistent form is a configuration choice (zx_tune compares it): pin it on the rings
    # used here, restore the defaults afterwards
    rings = (4096, 8192, 32768)
    before = {N: m.config_get(N) for N in rings}
    for N in rings:
        m.config_set(N, dict(before[N], fused=1))
    yield m
    for N in rings:
        m.config_set(N, before[N])


def flat_jobs(plan):
    """zx_transform_jobs' jobs launch by launch, each with its launch's ls and pass index."""
    out = []
    for k, launch in enumerate(plan["launches"]):
        for jd in launch["jobs"]:
            out.append(dict(jd, launch=k, ls=(jd["pad"] & 0xFF) or launch["ls"]))
    return out


def check_schedule_shape(sched, njobs):
    assert sorted(j for j, _ in sched) == list(range(njobs)), "the schedule is not a permutation of the jobs"
    for k, (_, deps) in enumerate(sched):
        assert all(0 <= d < k for d in deps), f"claim {k} waits for a job claimed later: {deps}"


def check_cell_order(sched, jobs):
    """Every store of a cell is ordered after the previous store and after the reads since it;
    every read after the store it reads. Accesses are taken launch by launch (jobs of one launch
    touch disjoint cells), which is the order of the per-pass form."""
    pos = {j: k for k, (j, _) in enumerate(sched)}
    deps = {j: set(d) for j, d in sched}
    claim_of = {k: j for k, (j, _) in enumerate(sched)}
    last_store, readers = {}, {}
    for j in sorted(range(len(jobs)), key=lambda t: (jobs[t]["launch"], t)):
        jd = jobs[j]
        need = set()
        for m, c in enumerate(job_cells(jd, max(jd["nload"], jd["nstore"]))):
            if c in last_store:
                need.add(last_store[c])
            if m < jd["nstore"]:
                need |= readers.get(c, set())
        got = {claim_of[d] for d in deps[j]}
        missing = need - got
        assert not missing, f"job {j} (claim {pos[j]}) does not wait for jobs {sorted(missing)[:8]}"
        for m, c in enumerate(job_cells(jd, max(jd["nload"], jd["nstore"]))):
            if m < jd["nstore"]:
                last_store[c] = j
                readers[c] = set()
            elif m < jd["nload"]:
                readers.setdefault(c, set()).add(j)


def replay(plan, sched, jobs, N, vals, L, order_seed, mode=0):
    """Run the jobs one at a time, each reading the buffer as the jobs before it left it: in the
    claim order (order_seed None) or in a random order among the jobs whose lists are done."""
    R = Fermat(N, mode)
    x = list(vals) + [0] * (L - len(vals))
    rng = random.Random(order_seed)
    done = [False] * len(sched)
    waiting = {k for k in range(len(sched))}
    while waiting:
        ready = [k for k in waiting if all(done[d] for d in sched[k][1])]
        assert ready, "no claimed job can run: the lists form a cycle"
        k = min(ready) if order_seed is None else rng.choice(ready)
        jd = jobs[sched[k][0]]
        cells = job_cells(jd, max(jd["nload"], jd["nstore"]))
        got = run_image(plan["images"][jd["image"]], jd["ls"], N, jd["e"], [x[c] for c in cells[:jd["nload"]]],
                        jd["nload"], jd["nstore"], jd["nscale"], jd["escale"], ring=R)
        for m, v in got.items():
            x[cells[m]] = v
        done[k] = True
        waiting.discard(k)
    return x


# (kind, l, z, n, f, e, N, scale): plans of two or more passes of single-CTA jobs (the persistent
# form exists for rings of four or more 32-bit words per lane, N >= 4096)
CASES = [
    (0, 10, 1024, 1024, 0, 17, 4096, 0),
    (1, 10, 1024, 1000, 1, 17, 4096, 0),
    (0, 11, 1500, 1999, 0, 3, 4096, 0),
    (1, 11, 1999, 1500, 1, 3, 4096, 1),
    (1, 11, 1025, 1025, 0, 0, 4096, 1),
    (0, 12, 2049, 2049, 0, 1, 4096, 0),
    (1, 12, 3001, 2999, 1, 5, 4096, 1),
    (0, 9, 300, 300, 0, 0, 4096, 0),
    (1, 9, 300, 300, 0, 0, 4096, 1),
    (0, 13, 5000, 6001, 0, 7, 8192, 0),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "k{}l{}z{}n{}f{}".format(*c[:5]))
def test_any_order_the_lists_allow_matches_the_oracle(tg, orc, case):
    kind, l, z, n, f, e, N, scale = case
    L = 1 << l
    p = (1 << N) + 1
    rng = random.Random(l * 131 + z)
    vals = [rng.randrange(p) for _ in range(z)]
    for i, v in zip(range(0, z, max(1, z // 3)), (0, p - 1, 1)):
        vals[i] = v
    plan = tg.transform_jobs(kind, l, z, n, N, f=f, e=e, scale=scale)
    sched = tg.transform_schedule(kind, l, z, n, N, f=f, e=e, scale=scale, slots=24)
    jobs = flat_jobs(plan)
    assert len(plan["launches"]) >= 2 and sched, "the case must have a persistent form"
    check_schedule_shape(sched, len(jobs))
    check_cell_order(sched, jobs)
    want = oracle_transform(orc, kind, vals, l, z, n, f, e, N, 0)
    if kind == 1 and scale:
        inv = pow(2, -l, p)
        want = [v * inv % p for v in want[:n]] + want[n:]
    outs = n if kind == 0 else n + f
    for seed in (None, 1, 2):
        got = replay(plan, sched, jobs, N, vals, L, seed)[:outs]
        assert got == want, (case, seed)


def test_the_benchmark_schedules_order_every_shared_cell(tg):
    """The l = 16, N = 32768 plans of the benchmark's n: one claim per job, every dependency
    claimed earlier, and each job waiting for the jobs that stored or read its cells before it."""
    for n in (32769, 40000, 52000, 65536):
        for kind in (0, 1):
            plan = tg.transform_jobs(kind, 16, n, n, 32768, scale=kind)
            sched = tg.transform_schedule(kind, 16, n, n, 32768, scale=kind)
            jobs = flat_jobs(plan)
            assert sched, (kind, n)
            check_schedule_shape(sched, len(jobs))
            check_cell_order(sched, jobs)


def test_the_schedule_interleaves_the_passes(tg):
    """The claim order takes the second pass of a top-level column while later columns are still
    in their first pass (so the second pass finds the cells in L2), rather than pass by pass."""
    plan = tg.transform_jobs(0, 16, 65536, 65536, 32768)
    sched = tg.transform_schedule(0, 16, 65536, 65536, 32768, slots=456)
    jobs = flat_jobs(plan)
    launches = [jobs[j]["launch"] for j, _ in sched]
    first_pass2 = launches.index(1)
    last_pass1 = len(launches) - 1 - launches[::-1].index(0)
    assert first_pass2 < 1000 < last_pass1, (first_pass2, last_pass1)


def test_cluster_small_ring_and_single_launch_plans_have_no_persistent_form(tg):
    # one launch (a transform that one job holds), rings of fewer than four words per lane, and
    # plans with cluster jobs keep their launches
    assert tg.transform_schedule(0, 6, 40, 37, 4096) == []
    assert tg.transform_schedule(0, 11, 2048, 2048, 1024) == []
    # N = 9216: sixteen words per lane in 18 of the 32 lanes; the persistent kernel is built for
    # rings that fill every lane only
    before = tg.config_get(9216)
    tg.config_set(9216, dict(before, fused=1))
    try:
        assert len(tg.transform_jobs(1, 11, 2048, 2000, 9216)["launches"]) >= 2
        assert tg.transform_schedule(1, 11, 2048, 2000, 9216) == []
    finally:
        tg.config_set(9216, before)
    N = 4096
    before = tg.config_get(N)
    tg.config_set(N, dict(ls_max=3, ls_c=3, max_warps=8, split=0, fused=1))
    try:
        plan = tg.transform_jobs(0, 12, 4096, 4096, N)
        assert any(L["lc"] > 0 for L in plan["launches"])
        assert tg.transform_schedule(0, 12, 4096, 4096, N) == []
        tg.config_set(N, dict(before, fused=0))
        assert tg.transform_schedule(0, 10, 1024, 1024, N) == []
    finally:
        tg.config_set(N, before)
