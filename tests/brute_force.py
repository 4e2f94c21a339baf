"""Brute-force enumeration of local alignments, used to pin the CPU oracle.

An alignment is a sequence of columns: M (query residue against reference
residue), I (query residue against a gap) and D (reference residue against a
gap).  A maximal run of L columns of the same gap kind costs ``gap_cost(L)``;
an I run directly followed by a D run (or the reverse) is two gaps.  A local
alignment that starts or ends with a gap scores strictly less than the same
alignment without it, so only alignments whose first and last columns are M
are enumerated.  Every such alignment of every substring pair is visited by a
depth-first walk; nothing is shared with the oracle's dynamic programme.
"""


def enumerate_local(q, r, score, gap_cost):
    """Yields (total, q_start, q_end, r_start, r_end) for every local alignment
    whose first and last columns are matches.

    q, r: sequences of codes; score(a, b): substitution score; gap_cost(L) > 0.
    """
    lq, lr = len(q), len(r)
    out = []

    def walk(i, j, last, run, gaps_closed, subst, qs, rs):
        # (i, j) is the last consumed cell; `last` is the kind of the last
        # column; `run` its current length when it is a gap.
        if last == "M":
            out.append((subst - gaps_closed, qs, i, rs, j))
            pending = 0
        else:
            pending = gap_cost(run)
        # M column
        if i + 1 < lq and j + 1 < lr:
            walk(i + 1, j + 1, "M", 0, gaps_closed + pending,
                 subst + score(q[i + 1], r[j + 1]), qs, rs)
        # I column (consumes a query residue)
        if i + 1 < lq:
            if last == "I":
                walk(i + 1, j, "I", run + 1, gaps_closed, subst, qs, rs)
            else:
                walk(i + 1, j, "I", 1, gaps_closed + pending, subst, qs, rs)
        # D column (consumes a reference residue)
        if j + 1 < lr:
            if last == "D":
                walk(i, j + 1, "D", run + 1, gaps_closed, subst, qs, rs)
            else:
                walk(i, j + 1, "D", 1, gaps_closed + pending, subst, qs, rs)

    for qs in range(lq):
        for rs in range(lr):
            walk(qs, rs, "M", 0, 0, score(q[qs], r[rs]), qs, rs)
    return out


def brute_record(q, r, score, gap_cost):
    """The record the oracle's conventions define, found by enumeration.

    score S = max(0, best total).  End: among optimal alignments, the smallest
    q_end, then the smallest r_end (row-major first).  Start: among optimal
    alignments ending there, the largest q_start, then the largest r_start.
    Also returns the set of all optimal (q_start, q_end, r_start, r_end).
    """
    alns = enumerate_local(q, r, score, gap_cost)
    best = max([a[0] for a in alns], default=0)
    if best <= 0:
        return (0, -1, -1, -1, -1), set()
    opt = {a[1:] for a in alns if a[0] == best}
    q_end, r_end = min((a[1], a[3]) for a in opt)
    starts = [(a[0], a[2]) for a in opt if a[1] == q_end and a[3] == r_end]
    q_start, r_start = max(starts)
    return (best, q_start, q_end, r_start, r_end), opt


def global_affine(q, r, score, go, ge):
    """Best global alignment score of q against r, gap of length L = go + ge*L.

    Plain three-state programme with gaps allowed at both ends; used to
    re-score a reported span.
    """
    NEG = -10 ** 9
    lq, lr = len(q), len(r)
    H = [[NEG] * (lr + 1) for _ in range(lq + 1)]
    E = [[NEG] * (lr + 1) for _ in range(lq + 1)]   # last column consumes r
    F = [[NEG] * (lr + 1) for _ in range(lq + 1)]   # last column consumes q
    H[0][0] = 0
    for j in range(1, lr + 1):
        E[0][j] = -(go + ge * j)
        H[0][j] = E[0][j]
    for i in range(1, lq + 1):
        F[i][0] = -(go + ge * i)
        H[i][0] = F[i][0]
    for i in range(1, lq + 1):
        for j in range(1, lr + 1):
            E[i][j] = max(E[i][j - 1] - ge, H[i][j - 1] - go - ge)
            F[i][j] = max(F[i - 1][j] - ge, H[i - 1][j] - go - ge)
            H[i][j] = max(H[i - 1][j - 1] + score(q[i - 1], r[j - 1]), E[i][j], F[i][j])
    return H[lq][lr]


def enumerate_global(q, r, score, go, ge):
    """Yields (total, identical columns, columns) for every global alignment
    of q against r: every sequence of columns D (q_i with r_j), V (q_i with a
    gap) and Z (a gap with r_j) consuming both; a maximal run of L gap
    columns of one kind costs go + ge * L.  For tiny inputs only."""
    lq, lr = len(q), len(r)

    def rec(i, j, last, run, total, same, cols):
        if i == lq and j == lr:
            closing = -(go + ge * run) if last in ("V", "Z") else 0
            yield total + closing, same, cols
            return
        def close():
            return -(go + ge * run) if last in ("V", "Z") else 0
        if i < lq and j < lr:
            yield from rec(i + 1, j + 1, "D", 0, total + close() + score(q[i], r[j]),
                           same + (q[i] == r[j]), cols + 1)
        if i < lq:
            if last == "V":
                yield from rec(i + 1, j, "V", run + 1, total, same, cols + 1)
            else:
                yield from rec(i + 1, j, "V", 1, total + close(), same, cols + 1)
        if j < lr:
            if last == "Z":
                yield from rec(i, j + 1, "Z", run + 1, total, same, cols + 1)
            else:
                yield from rec(i, j + 1, "Z", 1, total + close(), same, cols + 1)

    yield from rec(0, 0, None, 0, 0, 0, 0)


def enumerate_global_columns(q, r, score, go, ge):
    """Yields (total, columns) for every global alignment of q against r, the
    columns as a string over D (q_i with r_j), V (q_i with a gap) and Z (a gap
    with r_j); a maximal run of L gap columns of one kind costs go + ge * L.
    For tiny inputs only."""
    lq, lr = len(q), len(r)

    def rec(i, j, last, run, total, cols):
        closing = -(go + ge * run) if last in ("V", "Z") else 0
        if i == lq and j == lr:
            yield total + closing, cols
            return
        if i < lq and j < lr:
            yield from rec(i + 1, j + 1, "D", 0, total + closing + score(q[i], r[j]), cols + "D")
        if i < lq:
            if last == "V":
                yield from rec(i + 1, j, "V", run + 1, total, cols + "V")
            else:
                yield from rec(i + 1, j, "V", 1, total + closing, cols + "V")
        if j < lr:
            if last == "Z":
                yield from rec(i, j + 1, "Z", run + 1, total, cols + "Z")
            else:
                yield from rec(i, j + 1, "Z", 1, total + closing, cols + "Z")

    yield from rec(0, 0, None, 0, 0, "")


def preferred_alignment(optimal):
    """The one alignment the identity convention picks among the optimal
    global alignments `optimal` (column strings of equal score), chosen by
    the convention's own rule applied to the strings, walking back from the
    end: outside a gap, the last remaining column is a D if some optimal
    alignment has one there, else a V, else a Z; inside a gap run, the run
    starts at the current column (the column before it is of another kind)
    if some optimal alignment does so, else it extends one column further.
    Returns the column string."""
    rem = list(optimal)
    state = "H"
    picked = []
    while any(rem):
        if state == "H":
            for kind in "DVZ":
                cand = [s for s in rem if s.endswith(kind)]
                if cand:
                    break
            picked.append(kind)
            rem = [s[:-1] for s in cand]
            state = "H" if kind == "D" else kind
        else:
            opened = [s for s in rem if not s.endswith(state)]
            if opened:
                rem = opened
                state = "H"
            else:
                rem = [s[:-1] for s in rem]
                picked.append(state)
    return "".join(reversed(picked))


def identity_of(q, r, cols):
    """(identical columns, columns) of the alignment `cols` of q against r."""
    i = j = same = 0
    for c in cols:
        if c == "D":
            same += q[i] == r[j]
            i += 1
            j += 1
        elif c == "V":
            i += 1
        else:
            j += 1
    assert i == len(q) and j == len(r)
    return same, len(cols)
