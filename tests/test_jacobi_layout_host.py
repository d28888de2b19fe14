"""Host checks of the index design of the FP32 start block's Jacobi kernel
(cyclic Jacobi with the round-robin parallel ordering, Golub and Van Loan,
Matrix Computations, Sec. 8.5.5).

The kernel updates its shared-memory copy of B in place, one round at a time,
with no barrier between the blocks of a round. That is race-free only if:
- the wrapped half storage maps the unordered index pairs {i, j} of an m x m
  symmetric matrix one to one onto its slots;
- each round's pairs are disjoint and cover 0..M-1;
- the blocks (k, l), l >= k, of a round together touch every slot exactly
  once (the pair's own block writes its off-diagonal entry once).
These tests check the three properties for the kernel's index formulas,
restated here, over every order up to the kernel's largest (320), and every
round for a set of orders with both parities."""
import pytest

JACOBI_MAX = 320


def jacobi_ld(m):
    return (((m | 1) + 1) // 2 + 1) & ~1


def jacobi_slot(i, j, Mo, ld):
    d = j - i
    if d < 0:
        d += Mo
    return i * ld + d if d <= (Mo >> 1) else j * ld + (Mo - d)


def round_pairs(m, r):
    """Pairs (p, q), p < q, of round r of the tournament over M = m rounded up
    to even; q == m marks the idle index of an odd m."""
    M = m + (m & 1)
    out = []
    for t in range(M // 2):
        pa = 0 if t == 0 else 1 + (t - 1 + r) % (M - 1)
        k2 = M - 1 - t
        pb = 0 if k2 == 0 else 1 + (k2 - 1 + r) % (M - 1)
        out.append((min(pa, pb), max(pa, pb)))
    return out


@pytest.mark.parametrize("m", list(range(1, 66)) + [127, 128, 201, 202, 224, 255, 319, JACOBI_MAX])
def test_wrapped_storage_is_one_slot_per_entry(m):
    Mo, ld = m | 1, jacobi_ld(m)
    assert ld % 2 == 0 and ld >= (Mo + 1) // 2
    owner = {}
    for i in range(m):
        for j in range(m):
            s = jacobi_slot(i, j, Mo, ld)
            assert 0 <= s < m * ld
            assert owner.setdefault(s, (min(i, j), max(i, j))) == (min(i, j), max(i, j))
    assert len(owner) == m * (m + 1) // 2
    # the diagonal is column 0; the kernel's initial fill and norm loop walk
    # columns d < (Mo + 1) / 2 of each row and keep j = (i + d) mod Mo < m
    walked = set()
    for i in range(m):
        for d in range((Mo + 1) // 2):
            j = (i + d) % Mo
            if j < m:
                assert jacobi_slot(i, j, Mo, ld) == i * ld + d
                walked.add(i * ld + d)
    assert walked == set(owner)


def test_largest_order_fits_shared_memory():
    """B's slots and a 1/32 slab of the vectors, in FP32, stay within the
    227 KB a CTA may hold with the kernel's static arrays (2832 bytes)."""
    m = JACOBI_MAX
    cw = -(-m // min(32, m))
    assert 4 * (m * jacobi_ld(m) + m * cw) + 2832 <= 232448


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 8, 13, 32, 33, 64, 65, 97, 202])
def test_every_round_touches_each_slot_once(m):
    Mo, ld = m | 1, jacobi_ld(m)
    M = m + (m & 1)
    live = {jacobi_slot(i, j, Mo, ld) for i in range(m) for j in range(m)}
    for r in range(max(M - 1, 1)):
        pairs = round_pairs(m, r)
        flat = [x for pq in pairs for x in pq]
        assert sorted(flat) == list(range(M))  # disjoint, covering
        pp = [p for p, q in pairs]
        qq = [q if q < m else p for p, q in pairs]  # the idle pair rotates nothing
        count = {}
        half = len(pairs)
        for k in range(half):
            krot = qq[k] != pp[k]
            for l in range(k, half):
                lrot = qq[l] != pp[l]
                sa = jacobi_slot(pp[k], pp[l], Mo, ld)
                sb = jacobi_slot(pp[k], qq[l], Mo, ld)
                sd = jacobi_slot(qq[k], pp[l], Mo, ld)
                se = jacobi_slot(qq[k], qq[l], Mo, ld)
                writes = [sa]
                if l == k:
                    if krot:
                        assert sb == sd
                        writes += [sb, se]
                else:
                    if lrot:
                        writes.append(sb)
                    if krot:
                        writes.append(sd)
                        if lrot:
                            writes.append(se)
                for s in writes:
                    count[s] = count.get(s, 0) + 1
        assert set(count) == live and all(c == 1 for c in count.values()), (m, r)
