"""Shift-group partition of the phase average over ranks (one GPU per rank).

The Riemann terms w_m e^{-s_m L} N(e^{s_m L} U) of Eq. vt_discretised are
independent (Sec. 2.2); the paper distributes them over groups of processes
and reduces the groups' partial sums once (Sec. 2.5, last paragraph).  Here
rank g of G evaluates the contiguous group of shifts groups(M, G)[g] with
pavg_averaged_rhs_group (the shared-basis form restricted to the group, so a
group of small |s_m| runs a short Chebyshev chain), and one exchange step
follows: every rank gathers all G partial n-vectors and adds them in rank
order, so every rank holds the same, bitwise reproducible sum.

Host logic and one collective only: the arithmetic of each partial runs in
the library's kernels.
"""


def groups(M, G):
    """Contiguous groups [m0, m1) of the M shifts, sizes differing by at most one."""
    if G < 1 or M < G:
        raise ValueError("need 1 <= G <= M")
    return [(g * M // G, (g + 1) * M // G) for g in range(G)]


def reduce_partials(partial, dist=None):
    """Sum of every rank's partial vector, added in rank order (the result is
    identical on all ranks and independent of arrival order)."""
    if dist is None or dist.get_world_size() == 1:
        return partial
    parts = [partial.new_empty(partial.shape) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, partial.contiguous())
    out = parts[0].clone()
    for p in parts[1:]:
        out += p
    return out


def averaged_rhs(model, T, M, U, dist=None):
    """N-bar(U) by shift groups: this rank's group, then the one reduction."""
    rank = dist.get_rank() if dist is not None else 0
    world = dist.get_world_size() if dist is not None else 1
    m0, m1 = groups(M, world)[rank]
    return reduce_partials(model.averaged_rhs_group(T, M, m0, m1, U), dist)
