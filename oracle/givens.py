"""Greedy parallel annihilation schedule for the Givens RQ of a window block
(Algorithm 9, Sec. 3.2).  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The block is nRows x nCols with delta = nCols - nRows; row r (1-based) holds
its nonzeros in columns r .. nCols, and the RQ factorisation must zero the
entries (r, c) for r <= c < r + delta, so that row r keeps (r, r + delta)
and the first delta columns of the block vanish.  Entry (r, c1) is zeroed by a
rotation of columns c1 and c2 (c2 > c1, (r, c2) nonzero); rotations in one step
touch disjoint columns, so they can run concurrently.

Labels, as in Algorithm 9:
  ready      (r, c) in the band r <= c <= r + delta, not yet zeroed and not
             serving as a partner in the current step;
  available  may take part now: initially every entry of the bottom row and
             every diagonal entry (r, r) (the printed initialisation joins the
             two conditions with "and"; it is read as "or", the only reading
             that reproduces the paper's 13-step worked example); an entry
             above a zeroed one becomes
             available at the start of the step after that zeroing.
Each step scans the rows from the bottom; in row r, for c1 ascending, the first
ready-and-available (r, c1) is paired with the ready-and-available (r, c2)
with the largest c2 > c1; (r, c1) is then retired, (r, c2) is busy until the
step ends, and (r-1, c1) waits for the next step.  The loop ends with the first
step that schedules nothing, and every step found is executed (the loop of
Algorithm 10 is read as running over all of Algorithm 9's steps; stopping one
short would skip the last rotation of the worked example).
"""


def greedy_schedule(n_rows, n_cols, initial="bottom_or_diagonal"):
    """Return the list of steps; each step is a list of (r, c1, c2), 1-based.

    `initial` selects the reading of Algorithm 9's initialisation:
    "bottom_or_diagonal" (the "or" reading above) or "bottom_only" (the literal alternative, kept
    for the test that shows it does not reproduce the paper's figure).
    """
    delta = n_cols - n_rows
    if delta < 1 or n_rows < 1:
        return []
    band = {(r, c) for r in range(1, n_rows + 1) for c in range(r, r + delta + 1)}
    ready = set(band)
    if initial == "bottom_or_diagonal":
        available = {(r, c) for (r, c) in band if r == n_rows or c == r}
    elif initial == "bottom_only":
        available = {(r, c) for (r, c) in band if r == n_rows}
    else:
        raise ValueError(initial)
    busy = set()
    zeroed_last = []
    steps = []
    while True:
        # end of the previous step: partners return, entries above zeros open up
        ready |= busy
        busy = set()
        for (r, c) in zeroed_last:
            if r > 1:
                available.add((r - 1, c))
        zeroed_last = []
        step = []
        for r in range(n_rows, 0, -1):
            for c1 in range(r, r + delta + 1):
                if (r, c1) in ready and (r, c1) in available:
                    for c2 in range(r + delta, c1, -1):
                        if (r, c2) in ready and (r, c2) in available:
                            step.append((r, c1, c2))
                            ready.discard((r, c1))
                            ready.discard((r, c2))
                            busy.add((r, c2))
                            if r > 1:
                                available.discard((r - 1, c1))
                            zeroed_last.append((r, c1))
                            break
        if not step:
            return steps
        steps.append(step)
