"""Level schedules and table sizes (oracle; test infrastructure only).

Levels are returned COARSE -> FINE as a list of [Rx, Ry, Rz, Rt] vertex counts.
The paper numbers its levels the other way (level 1 = finest, Eq. 4).
"""
import math


def ceil_log(f, s):
    """ceil(log_f s) for integers, exactly: the smallest L >= 0 with f**L >= s (Eq. 5)."""
    L, p = 0, 1
    while p < s:
        p *= f
        L += 1
    return L


def fold_schedule(S, St, fold, rule="max"):
    """Fold policy of Section 3.2.1 (Eqs. 4-8) and its temporal use in Section 3.2.2.

    S = (Sx, Sy, Sz): native FBB resolution (level 1, Eq. 4); St: number of key frames
    (the temporal native resolution).  L_d = ceil(log_f S_d) (Eq. 5); the shared level count
    L_s is their maximum (Eq. 6, rule "max") or, reading Table 3's "Res level", their
    minimum (rule "min").  Each further level divides the previous resolution by f, rounding
    up, while it exceeds f; otherwise it takes the tail value 2 (Eqs. 7-8).  The same
    recursion runs on the time axis over the same L_s levels.
    """
    if fold < 2:
        raise ValueError("fold must be >= 2")
    Ls = [ceil_log(fold, s) for s in S]
    L = max(Ls) if rule == "max" else min(Ls)
    L = max(L, 1)
    levels = [[int(S[0]), int(S[1]), int(S[2]), int(St)]]           # level 1, Eq. 4
    for _ in range(2, L + 1):
        prev = levels[-1]
        levels.append([-(-r // fold) if r > fold else 2 for r in prev])  # Eq. 7 / Tail(l) = 2
    return levels[::-1]


def geometric_schedule(r0, r1, L):
    """R_l = floor(r0 * (r1/r0)**(l/(L-1)) + 0.5) per axis, l = 0..L-1 (double precision)."""
    out = []
    for l in range(L):
        row = []
        for d in range(4):
            if L == 1:
                row.append(int(r1[d]))
            else:
                row.append(int(math.floor(r0[d] * (r1[d] / r0[d]) ** (l / (L - 1)) + 0.5)))
        out.append(row)
    return out


def level_rows(R):
    """Number of table rows of one level: every vertex of the Rx x Ry x Rz x Rt grid (Eq. 9 is a
    bijection onto [0, Rx*Ry*Rz*Rt))."""
    return int(R[0]) * int(R[1]) * int(R[2]) * int(R[3])


def bases(levels):
    """Row offset of each level in the concatenated table, and the total row count."""
    b, acc = [], 0
    for R in levels:
        b.append(acc)
        acc += level_rows(R)
    return b, acc


def param_count(levels, F, mlp_dims=None):
    """Encoding parameters (rows x F), plus MLP weights and biases when dims are given."""
    n = bases(levels)[1] * F
    if mlp_dims:
        n += sum(mlp_dims[k] * mlp_dims[k + 1] + mlp_dims[k + 1] for k in range(len(mlp_dims) - 1))
    return n
