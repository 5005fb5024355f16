"""External-row order of the classes, rebuilt in plain Python from the
convention e2.h documents for e2_partials (test helper; no GPU, no product
code): pairs x < y have index y(y-1)/2 + x over the correlated virtual (or
core) spinors; (i, a<b) is i * npair_v + pair(a,b); (i<j, a) is
pair(i,j) * n_vc + a; (i, a) is i * n_vc + a; (i<j) is pair(i,j)."""


def _pair(e):
    """(x, y), x < y, of pair index e = y(y-1)/2 + x."""
    y = int((1 + (1 + 8 * e) ** 0.5) / 2)
    while y * (y - 1) // 2 > e:
        y -= 1
    while (y + 1) * y // 2 <= e:
        y += 1
    return e - y * (y - 1) // 2, y


# class id -> (h, p); rows decoded per e2.h's documented order
CLASSES = {2: (0, 2), 5: (1, 2), 7: (2, 1), 4: (1, 1), 6: (2, 0), 1: (0, 1), 3: (1, 0), 0: (0, 0)}


def _row(cls, row, cc, vc):
    """(holes, particles) as global spinor indices of external row `row`."""
    nvc, nvp = len(vc), len(vc) * (len(vc) - 1) // 2
    if cls == 2:
        a, b = _pair(row)
        return [], [vc[a], vc[b]]
    if cls == 5:
        a, b = _pair(row % nvp)
        return [cc[row // nvp]], [vc[a], vc[b]]
    if cls == 7:
        i, j = _pair(row // nvc)
        return [cc[i], cc[j]], [vc[row % nvc]]
    if cls == 4:
        return [cc[row // nvc]], [vc[row % nvc]]
    if cls == 6:
        i, j = _pair(row)
        return [cc[i], cc[j]], []
    if cls == 1:
        return [], [vc[row]]
    if cls == 3:
        return [cc[row]], []
    if cls == 0:
        return [], []
    raise ValueError(cls)
