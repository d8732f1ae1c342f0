"""Execution of job images on Python values: the schedule the GPU kernel runs, checked
without a GPU. A job image lists, per cluster CTA and stage, the base-case butterflies of
Algorithms 1 and 2 (Secs. 3-4) on shared-memory slots, plus the layout exchanges between the
CTAs of a cluster. A cell is a value x with a pending rotation t (it stands for x omega^t).
Test infrastructure: the format mirrors the kernel's job image words, the arithmetic is plain
Python integers."""

OP_BF, OP_CROSS, OP_TAG = 1, 2, 3
OPF_S, OPF_D, OPF_S_TO_J, OPF_D_TO_I, OPF_COPY = 1, 2, 4, 8, 16
STAGE_PROG, STAGE_XCHG, STAGE_SWAP = 0, 1, 2


def job_cell(layout, rank, slot, C, L2, b):
    if C == 1:
        return slot
    if layout == 0:
        return rank * L2 + slot
    return (slot // b) * L2 + rank * b + slot % b


def ops_of(img, off):
    nlev = int(img[off])
    nops = int(img[off + 1])
    starts = [int(v) for v in img[off + 2:off + 3 + nlev]]
    base = off + ((3 + nlev + 1) & ~1)
    ops = []
    for k in range(nops):
        w = [int(v) for v in img[base + 10 * k:base + 10 * k + 10]]
        ops.append(dict(i=w[0] & 0xFFFF, j=w[0] >> 16, kind=w[1] & 0xFF, flags=(w[1] >> 8) & 0xFF,
                        scal=w[1] >> 16, ra=(w[2], w[3]), rb=(w[4], w[5]), p0=(w[6], w[7]), p1=(w[8], w[9])))
    return starts, ops


OPS_A_DOUBLE, OPS_A_HALVE, OPS_S_HALVE = 1, 2, 4


class Fermat:
    """Z/(2^N+1) with omega = 2 (mode 0) or omega = sqrt2 (mode 2); values are ints."""

    def __init__(self, N, mode=0):
        self.p, self.order = (1 << N) + 1, (4 if mode == 2 else 2) * N
        self.w = ((1 << (3 * N // 4)) - (1 << (N // 4))) % self.p if mode == 2 else 2
        self.zero = 0

    def pow(self, v, t):
        return v * pow(self.w, t % self.order, self.p) % self.p

    def add(self, a, b):
        return (a + b) % self.p

    def sub(self, a, b):
        return (a - b) % self.p

    def scale(self, v, k):  # times 2^k, k in {-1, 1}
        return v * pow(2, k, self.p) % self.p


class SnRing:
    """S[y]/(y^H+1), S = Z/mZ (mode 1); values are tuples of H ints."""

    def __init__(self, H, m):
        self.H, self.m, self.order = H, m, 2 * H
        self.zero = (0,) * H

    def pow(self, v, t):
        t %= self.order
        neg = t >= self.H
        t -= self.H if neg else 0
        out = [0] * self.H
        for i, c in enumerate(v):
            j, c2 = i + t, c
            if j >= self.H:
                j, c2 = j - self.H, -c
            out[j] = (-c2 if neg else c2) % self.m
        return tuple(out)

    def add(self, a, b):
        return tuple((x + y) % self.m for x, y in zip(a, b))

    def sub(self, a, b):
        return tuple((x - y) % self.m for x, y in zip(a, b))

    def scale(self, v, k):
        f = pow(2, k, self.m)
        return tuple(x * f % self.m for x in v)


def run_image(img, ls, N, e, inputs, nload, nstore, nscale=0, escale=0, ring=None):
    """Execute a job image on Python values (ints mod 2^N+1 unless `ring` says otherwise);
    returns the stored cell values {cell: value}. Scalar flags (mode 1) are applied as read."""
    R = ring or Fermat(N)
    twoN = R.order
    nst, C, load_l, store_l = (int(v) for v in img[:4])
    lc = C.bit_length() - 1
    nslots = 1 << (ls - lc)
    L2, b = nslots, nslots // C
    rot = lambda a: (a[0] * e + a[1]) % twoN
    state = [[(R.zero, 0)] * nslots for _ in range(C)]
    for c in range(C):
        for s in range(nslots):
            m = job_cell(load_l, c, s, C, L2, b)
            state[c][s] = (inputs[m] if m < nload else R.zero, 0)
    for st in range(nst):
        ent = 4 + st * (2 + C)
        typ, arg = int(img[ent]), int(img[ent + 1])
        if typ == STAGE_PROG:
            for c in range(C):
                off = int(img[ent + 2 + c])
                if not off:
                    continue
                starts, ops = ops_of(img, off)
                sc = state[c]
                for v in range(len(starts) - 1):
                    touched = set()
                    for o in ops[starts[v]:starts[v + 1]]:
                        for cell in {o["i"], o["j"]}:
                            assert cell not in touched, "ops of one level share a cell"
                            touched.add(cell)
                        xi, ti = sc[o["i"]]
                        xj, tj = sc[o["j"]]
                        sa = 1 if o["scal"] & OPS_A_DOUBLE else (-1 if o["scal"] & OPS_A_HALVE else 0)
                        if o["kind"] == OP_TAG:
                            if o["flags"] & OPF_COPY:
                                sc[o["j"]] = (xi, (ti + rot(o["rb"])) % twoN)
                            sc[o["i"]] = (R.scale(xi, sa) if sa else xi, (ti + rot(o["ra"])) % twoN)
                            continue
                        A = R.pow(xi, ti + rot(o["ra"]))
                        if sa:
                            A = R.scale(A, sa)
                        B = R.pow(xj, tj + rot(o["rb"]))
                        if o["kind"] == OP_BF:
                            if o["flags"] & OPF_S:
                                dst = o["j"] if o["flags"] & OPF_S_TO_J else o["i"]
                                S = R.add(A, B)
                                sc[dst] = (R.scale(S, -1) if o["scal"] & OPS_S_HALVE else S, rot(o["p0"]))
                            if o["flags"] & OPF_D:
                                dst = o["i"] if o["flags"] & OPF_D_TO_I else o["j"]
                                sc[dst] = (R.sub(A, B), rot(o["p1"]))
                        else:
                            D = R.sub(A, B)
                            sc[o["j"]] = (D, rot(o["p1"]))
                            sc[o["i"]] = (R.add(A, D), 0)
        else:
            only = arg if typ == STAGE_SWAP else -1
            new = [list(row) for row in state]
            for x in range(C):
                for y in range(C):
                    if y == x or not (only < 0 or x == only or y == only):
                        continue
                    for i in range(b):
                        new[x][y * b + i] = state[y][x * b + i]
            state = new
    out = {}
    for c in range(C):
        for s in range(nslots):
            m = job_cell(store_l, c, s, C, L2, b)
            if m < nstore:
                x, t = state[c][s]
                t += escale if m < nscale else 0
                out[m] = R.pow(x, t)
    return out
