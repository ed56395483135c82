"""Shared-memory bank model of the pencil-task Picard sweeps (picard_pt in adg_kernels.cuh).

Counts the shared-memory wavefronts of one time slice of one block: the node threads' flux
stores and derivative loads (one 4-byte access per node and flux component), and the tasks'
pencil loads and derivative stores (n per task; 8-byte accesses where the x direction is stored
pencil-major and n is even).  A 4-byte warp access costs as many wavefronts as the largest
number of distinct words that map to one of the 32 banks; an 8-byte access is served per
half-warp.  For each configuration it searches the layout (PtLayout in adg_kernels.cuh):

  xpm   0: every direction position-major, value (p, m) at p + m MS
        1: x pencil-major (p SF0 + m), y and z position-major
  ord1  numbering of the y pencils: 0 p = x + n z, 1 p = z + n x
  MS    stride of the position along a direction (>= NP)
  CS    values per flux component and cell

and prints the best against the ideal (no conflicts).  pt_layout in adg_kernels.cuh holds these
results for the configurations the library builds; others use xpm = 0, ord1 = 0, MS = NP + 2.
check() replays the kernel's index arithmetic for a layout (bounds, coverage, alignment),
check_final() the final stage's trace stores, check_schedule() the double-buffered phases.
node_order() and x_task_order() build the thread orders of the nodes and of the x tasks that
make the 3D Euler N=5 accesses conflict-free (kNodeOrderEuler3N5 and kXTaskOrderEuler3N5 in
adg_kernels.cuh); count() takes them as optional arguments.

    python tests/pencil_layout_model.py
"""
import itertools


def wavefronts32(addrs):
    banks = {}
    for a in addrs:
        if a is not None:
            banks.setdefault(a % 32, set()).add(a)
    return max((len(s) for s in banks.values()), default=0)


def wavefronts64(addrs):
    total = 0
    for half in (addrs[:16], addrs[16:]):
        banks = {}
        for a in half:
            if a is not None:
                for w in (a, a + 1):
                    banks.setdefault(w % 32, set()).add(w)
        total += max((len(s) for s in banks.values()), default=0)
    return total


class Config:
    def __init__(self, name, D, n, V, nz):
        self.name, self.D, self.n, self.V, self.nz = name, D, n, V, nz
        self.NS, self.NP = n ** D, n ** (D - 1)
        self.CPB = 1 if self.NS >= 96 else 128 // self.NS
        self.THREADS = self.CPB * self.NS
        # flux components with a nonzero flux, direction-major ("combos")
        self.combos = [(d, v) for d in range(D) for v in range(V) if nz(d, v)]
        self.dir_of = [d for d, _ in self.combos]
        self.NC = len(self.dir_of)
        self.SF0 = n if n % 2 == 0 else n + 1

    def pencil(self, i, d, ord1):
        n = self.n
        x, y, z = i % n, (i // n) % n, i // (n * n)
        if d == 0:
            return y + n * z, x
        if d == 1:
            return (z + n * x) if ord1 else (x + n * z), y
        return x + n * y, z

    def addr(self, lay, cl, c, p, m):
        xpm, ord1, MS, CS = lay
        off = p * self.SF0 + m if (xpm and self.dir_of[c] == 0) else p + m * MS
        return cl * self.NC * CS + c * CS + off

    def slots(self, lay, xorder=None):
        """Task slots as the kernel assigns them: with xpm, slot j holds the tasks of direction j
        (thread i takes task i of that direction, or task xorder[i] of the x direction);
        otherwise slot j holds task i + j THREADS of the combo-major list.  Yields (slot,
        [(cell, combo, pencil) or None per thread])."""
        xpm = lay[0]
        NP, TH, CPB = self.NP, self.THREADS, self.CPB
        if xpm:
            for j in range(self.D):
                combos = [c for c in range(self.NC) if self.dir_of[c] == j]
                nt = len(combos) * NP
                task = (lambda t: xorder[t]) if (j == 0 and xorder is not None) else (lambda t: t % nt)
                yield j, [(t // nt, combos[task(t) // NP], task(t) % NP) if t < CPB * nt else None
                          for t in range(TH)]
        else:
            NT = self.NC * NP
            for j in range((CPB * NT + TH - 1) // TH):
                yield j, [((t // NT), (t % NT) // NP, t % NP) if t < CPB * NT else None
                          for t in (i + j * TH for i in range(TH))]

    def node_off(self, lay, i, d):
        """Offset of node i inside a combo region of direction d (the kernel's node_off)."""
        xpm, ord1, MS, CS = lay
        p, m = self.pencil(i, d, ord1)
        return p * self.SF0 + m if (xpm and d == 0) else p + m * MS

    def node_of(self, tid, order=None):
        """Node of thread tid in its cell: the identity, or order[tid] (one cell per block)."""
        return tid % self.NS if order is None else order[tid]

    def count_nodes(self, lay, order=None):
        """Wavefronts of the node threads' accesses, one flux component of each combo."""
        ord1 = lay[1]
        node = 0
        for w in range(0, self.THREADS, 32):
            lanes = [w + l if w + l < self.THREADS else None for l in range(32)]
            for c in range(self.NC):
                d = self.dir_of[c]
                node += wavefronts32([None if t is None else
                                      self.addr(lay, t // self.NS, c, *self.pencil(self.node_of(t, order), d, ord1))
                                      for t in lanes])
        return node

    def count(self, lay, order=None, xorder=None):
        xpm, ord1, MS, CS = lay
        node = self.count_nodes(lay, order)
        tasks = 0
        for j, tl in self.slots(lay, xorder):
            for w in range(0, self.THREADS, 32):
                cp = tl[w:w + 32] + [None] * max(0, w + 32 - self.THREADS)
                if all(x is None for x in cp):
                    continue
                pm = [x if (x and xpm and self.dir_of[x[1]] == 0) else None for x in cp]
                po = [x if (x and not (xpm and self.dir_of[x[1]] == 0)) else None for x in cp]
                if any(pm):
                    if self.n % 2 == 0:
                        for m in range(0, self.n, 2):
                            tasks += wavefronts64([None if x is None else self.addr(lay, *x, m) for x in pm])
                    else:
                        for m in range(self.n):
                            tasks += wavefronts32([None if x is None else self.addr(lay, *x, m) for x in pm])
                if any(po):
                    for m in range(self.n):
                        tasks += wavefronts32([None if x is None else self.addr(lay, *x, m) for x in po])
        # fluxes and derivatives share the layout: stores and loads cost the same
        return 2 * (node + tasks)

    def node_order(self, lay):
        """A thread -> node order (one cell per block) in which the nodes of every warp fall in 32
        distinct banks in every direction's region.  Node t goes to lane t mod 32, so a direction
        whose node offset is congruent to t mod 32 is conflict-free in any such order; the one
        other direction's offsets f(t) are handled as an edge colouring of the bipartite
        multigraph with an edge (t mod 32, f(t) mod 32) per node: every warp takes a matching.
        With W warps and r lanes in the last, residues below r have W nodes and the others W - 1;
        when f's residues have W or W - 1 nodes as well, the last warp takes a perfect matching
        of the W-node residues of both sides, after which the multigraph is (W - 1)-regular and
        splits into W - 1 perfect matchings (Koenig's theorem), found one by one by augmenting
        paths.  Among equal choices a node stays in its own warp.  Returns order (thread -> node)
        or None when the layout is not of this kind."""
        if self.CPB != 1 or self.D != 3:
            return None
        ord1 = lay[1]
        NS = self.NS
        offs = [[self.node_off(lay, t, d) for t in range(NS)] for d in range(self.D)]
        other = [d for d in range(self.D) if any((offs[d][t] - t) % 32 for t in range(NS))]
        if len(other) != 1:
            return None
        f = [o % 32 for o in offs[other[0]]]
        W = (NS + 31) // 32
        r = NS - 32 * (W - 1)
        cnt = [f.count(b) for b in range(32)]
        if any(c not in (W - 1, W) for c in cnt):
            return None
        edges = {}
        for t in range(NS):
            edges.setdefault((t % 32, f[t]), []).append(t)

        def matching(w, left, right):
            adj = {}
            for a in left:
                own = [b for b in right if any(t // 32 == w for t in edges.get((a, b), []))]
                adj[a] = own + [b for b in right if edges.get((a, b)) and b not in own]
            match = {}

            def augment(a, seen):
                for b in adj[a]:
                    if b not in seen:
                        seen.add(b)
                        if b not in match or augment(match[b], seen):
                            match[b] = a
                            return True
                return False

            for a in left:
                if not augment(a, set()):
                    raise AssertionError("no perfect matching")
            picked = []
            for b, a in match.items():
                ts = edges[(a, b)]
                t = next((t for t in ts if t // 32 == w), ts[0])
                ts.remove(t)
                picked.append(t)
            return picked

        groups = [None] * W
        groups[W - 1] = matching(W - 1, [a for a in range(32) if a < r],
                                 [b for b in range(32) if cnt[b] == W])
        for w in range(W - 1):
            groups[w] = matching(w, list(range(32)), list(range(32)))
        order = [None] * NS
        for w, g in enumerate(groups):
            for t in g:
                order[32 * w + t % 32] = t
        assert sorted(order) == list(range(NS))
        return order

    def x_task_order(self, lay):
        """A thread order of the x tasks (x pencil-major layouts, one cell per block, even n) in
        which every half-warp's 8-byte accesses fall in 16 distinct bank pairs.  The pair of task
        i is (its first value's word / 2) mod 16, the same for every position; if the H half-warps
        of the x slot find every pair class of size H - 1 or H, half-warp h < H - 1 takes the h-th
        task of each class (lane = class) and the last takes the last task of each class of size
        H.  Returns order (thread -> task of the x direction) or None."""
        if not lay[0] or self.CPB != 1 or self.n % 2:
            return None
        c0, NP = self.dir_of.index(0), self.NP
        nt = self.dir_of.count(0) * NP
        pair = [(self.addr(lay, 0, c0 + i // NP, i % NP, 0) // 2) % 16 for i in range(nt)]
        classes = [[i for i in range(nt) if pair[i] == r] for r in range(16)]
        H = (nt + 15) // 16
        if any(len(k) not in (H - 1, H) for k in classes):
            return None
        order = [classes[t % 16][t // 16] for t in range(16 * (H - 1))]
        order += [k[H - 1] for k in classes if len(k) == H]
        assert sorted(order) == list(range(nt))
        return order

    def check(self, lay, xorder=None):
        """The kernel's index arithmetic for layout lay, replayed: every node writes its own slot
        of each flux component inside its cell's region; the tasks of all threads read exactly the
        slots the nodes write and write (once each) exactly the slots the nodes read; 8-byte task
        accesses are aligned.  Slots: with xpm, slot j holds the tasks of direction j (thread i takes
        task i); otherwise slot j holds task i + j THREADS.  Raises AssertionError on a violation."""
        xpm, ord1, MS, CS = lay
        n, NP, NS, CPB, TH = self.n, self.NP, self.NS, self.CPB, self.THREADS
        assert MS >= NP and CS % 4 == 0 and CS >= (n - 1) * MS + NP and (not xpm or CS >= NP * self.SF0)
        assert self.D == 3 or (not xpm and not ord1)
        CELL = self.NC * CS
        written = set()
        for tid in range(TH):
            cl, i = tid // NS, tid % NS
            for c in range(self.NC):
                a = self.addr(lay, cl, c, *self.pencil(i, self.dir_of[c], ord1))
                assert cl * CELL + c * CS <= a < cl * CELL + (c + 1) * CS and a not in written
                written.add(a)
        cstart = [self.dir_of.index(d) for d in range(self.D)]
        ncd = [self.dir_of.count(d) for d in range(self.D)]
        NT = self.NC * NP
        nslot = self.D if xpm else (CPB * NT + TH - 1) // TH
        if xpm:
            assert all(CPB * k * NP <= TH for k in ncd)
        read, wrote = set(), set()
        for tid in range(TH):
            for j in range(nslot):
                # the kernel's task_base(j)
                if xpm:
                    nt = ncd[j] * NP
                    if tid >= CPB * nt:
                        continue
                    cl, r = tid // nt, tid % nt
                    if j == 0 and xorder is not None:
                        r = xorder[tid]
                    c, p = cstart[j] + r // NP, r % NP
                    base, stride = cl * CELL + c * CS + (p * self.SF0 if j == 0 else p), (1 if j == 0 else MS)
                    if j == 0 and n % 2 == 0:
                        assert base % 2 == 0
                else:
                    t = tid + j * TH
                    if t >= CPB * NT:
                        assert j == nslot - 1
                        continue
                    cl, r = t // NT, t % NT
                    base, stride = cl * CELL + (r // NP) * CS + r % NP, MS
                for m in range(n):
                    a = base + m * stride
                    assert a in written and a not in wrote
                    read.add(a)
                    wrote.add(a)
        assert read == written and wrote == written
        return True

    def node_of_face(self, d, j, a):
        n = self.n
        if self.D == 2:
            return a + n * j if d == 0 else j + n * a
        if d == 0:
            return a + n * j
        if d == 1:
            return (j % n) + n * (a + n * (j // n))
        return j + n * n * a

    def face_of(self, lay, d, p):
        n = self.n
        return p // n + n * (p % n) if (d == 1 and lay[1]) else p

    def check_final(self, lay, xorder=None):
        """The final stage's trace stores, replayed: the face index of every task's pencil names
        the same nodes (node_of_face), and every trace value of every cell, [dir][side][Qbar, Fbar.n]
        [v][face node], is written exactly once (Fbar.n by the Fbar tasks, Qbar and the Fbar.n of
        vanishing flux components by the Qbar tasks).  Raises AssertionError on a violation."""
        xpm, ord1, MS, CS = lay
        n, NP, NS, TH, CPB, D, V = self.n, self.NP, self.NS, self.THREADS, self.CPB, self.D, self.V
        NF = NP
        for i in range(NS):
            for d in range(D):
                p, m = self.pencil(i, d, ord1)
                assert self.node_of_face(d, self.face_of(lay, d, p), m) == i
        count = {}
        for j, tl in self.slots(lay, xorder):
            for x in tl:
                if x is None:
                    continue
                cl, c, p = x
                d, v = self.combos[c]
                for side in (0, 1):
                    key = (cl, d, side, 1, v, self.face_of(lay, d, p))
                    count[key] = count.get(key, 0) + 1
        NQ = CPB * D * V * NF
        for t in range(NQ):
            cl, r = t // (D * V * NF), t % (D * V * NF)
            d, v, jf = r // (V * NF), (r // NF) % V, r % NF
            for side in (0, 1):
                for qf in ((0, 1) if not self.nz(d, v) else (0,)):
                    key = (cl, d, side, qf, v, jf)
                    count[key] = count.get(key, 0) + 1
        want = {(cl, d, side, qf, v, jf) for cl in range(CPB) for d in range(D) for side in (0, 1)
                for qf in (0, 1) for v in range(V) for jf in range(NF)}
        assert set(count) == want and all(k == 1 for k in count.values())
        return True

    def ideal(self):
        return 2 * (self.NC * self.THREADS / 32 + self.CPB * self.NC * self.NP * self.n / 32)

    def search(self):
        best = None
        for xpm, ord1 in itertools.product((0, 1) if self.D == 3 else (0,), (0, 1) if self.D == 3 else (0,)):
            for MS in range(self.NP, self.NP + 8):
                ext = (self.n - 1) * MS + self.NP
                if xpm:
                    ext = max(ext, self.NP * self.SF0)
                for CS in range((ext + 3) // 4 * 4, (ext + 3) // 4 * 4 + 48, 4):
                    lay = (xpm, ord1, MS, CS)
                    if xpm and any(self.CPB * self.dir_of.count(d) * self.NP > self.THREADS for d in range(self.D)):
                        continue
                    w = self.count(lay)
                    if best is None or w < best[0]:
                        best = (w, lay)
        return best


def check_schedule(n, iters):
    """Replays the phases of picard_pt (barriers between phases) with two flux buffers F0, F1 and
    two derivative buffers R0, R1, each holding the tag (sweep, slice) of its last write.  Asserts
    that every read sees the slice it means to, and that no buffer is read and written in one
    phase (so a barrier always separates a write from the reads before and after it)."""
    buf = {}
    phases = []

    def phase(ops):
        reads = {b for op, b, _ in ops if op == "r"}
        writes = {b for op, b, _ in ops if op == "w"}
        assert not reads & writes, ops
        for op, b, tag in ops:
            if op == "r":
                assert buf.get(b) == tag, (b, buf.get(b), tag)
        for op, b, tag in ops:
            if op == "w":
                buf[b] = tag
        phases.append(ops)

    F = lambda k: "F%d" % (k % 2)
    R = lambda k: "R%d" % (k % 2)
    if iters <= 0:
        return 0
    phase([("w", "F0", (0, 0))])                                   # first sweep: one slice
    phase([("r", "F0", (0, 0)), ("w", "R0", (0, 0))])              # its tasks
    pending = [("r", "R0", (0, 0))]                                # q = Q - dt rowsum(P) R
    for r in range(1, iters):
        phase(pending + [("w", "F0", (r, 0))])
        for k in range(1, n + 1):
            ops = [("r", F(k - 1), (r, k - 1)), ("w", R(k - 1), (r, k - 1))]
            if k < n:
                ops.append(("w", F(k), (r, k)))
            if k >= 2:
                ops.append(("r", R(k), (r, k - 2)))
            phase(ops)
        pending = [("r", R(n - 1), (r, n - 1))]
    phase(pending)                                                 # the final stage follows
    return len(phases) - 1                                         # barriers


# the nonzero flux components of the PDEs built with an FP32 predictor (Phys::nz)
ALL = lambda d, v: True
ACOUSTIC = lambda d, v: v == 0 or v == 1 + d
ELASTIC3 = lambda d, v: not ((d == 0 and v == 4) or (d == 1 and v == 5) or (d == 2 and v == 3))
CONFIGS = [
    Config("acoustic 2D N=3", 2, 4, 3, ACOUSTIC),
    Config("acoustic 2D N=2", 2, 3, 3, ACOUSTIC),
    Config("acoustic 3D N=4", 3, 5, 4, ACOUSTIC),
    Config("acoustic 3D N=2", 3, 3, 4, ACOUSTIC),
    Config("elastic 3D N=6", 3, 7, 9, ELASTIC3),
    Config("elastic 3D N=2", 3, 3, 9, ELASTIC3),
    Config("elastic 2D N=3", 2, 4, 5, ALL),
    Config("Euler 3D N=5", 3, 6, 5, ALL),
    Config("Euler 3D N=2", 3, 3, 5, ALL),
    Config("Euler 2D N=5", 2, 6, 4, ALL),
    Config("Euler 2D N=3", 2, 4, 4, ALL),
    Config("shallow water N=4", 2, 5, 3, ALL),
    Config("shallow water N=2", 2, 3, 3, ALL),
]

if __name__ == "__main__":
    for cfg in CONFIGS:
        default = (0, 0, cfg.NP + 2, ((cfg.n - 1) * (cfg.NP + 2) + cfg.NP + 3) // 4 * 4)
        w, lay = cfg.search()
        order = cfg.node_order(lay)
        xorder = cfg.x_task_order(lay) if order is not None else None
        ordered = f", {cfg.count(lay, order, xorder)} in thread order" if order is not None else ""
        print(f"{cfg.name:18s} D={cfg.D} n={cfg.n} combos={cfg.NC:2d}: best xpm={lay[0]} ord1={lay[1]} "
              f"MS={lay[2]} CS={lay[3]}: {w} wavefronts{ordered} (default {cfg.count(default)}, "
              f"ideal {cfg.ideal():.0f})", flush=True)
