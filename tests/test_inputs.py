"""Structural checks of the seeded input generator (tree encoding, ordering)."""
import numpy as np

from paper_2202_06088_gb300 import inputs as I


def _walk(st):
    """Recover (level, coords) of every leaf by walking the child table."""
    found = {}
    stack = [(0, 0, (0, 0, 0))]
    while stack:
        node, L, c = stack.pop()
        for slot in range(8):
            e = int(st.child[node * 8 + slot])
            cc = (2 * c[0] + (slot >> 2 & 1), 2 * c[1] + (slot >> 1 & 1), 2 * c[2] + (slot & 1))
            if e == 0xFFFFFFFF:
                continue
            if e & 0x80000000:
                found[e & 0x7FFFFFFF] = (L + 1, cc)
            else:
                assert e > node
                stack.append((e, L + 1, cc))
    return found


def test_child_table_encodes_the_leaves():
    for seed in range(4):
        st = I.random_mixed_tree(4, seed)
        found = _walk(st)
        assert len(found) == st.n_leaves
        for i, (L, c) in found.items():
            assert st.leaf_level[i] == L and tuple(st.leaf_coords[i]) == c


def test_breadth_first_node_order_and_morton_leaf_order():
    st = I.random_mixed_tree(5, 11)
    # children of a node at level L have indices above every level-L node
    levels = np.zeros(st.n_nodes, int)
    for n in range(st.n_nodes):
        for s in range(8):
            e = int(st.child[n * 8 + s])
            if e != 0xFFFFFFFF and not e & 0x80000000:
                levels[e] = levels[n] + 1
    assert np.all(np.diff(levels) >= 0)
    fine = st.leaf_coords.astype(np.int64) << (st.depth - st.leaf_level)[:, None]
    assert np.all(np.diff(I.morton3(fine)) > 0)


def test_config1_scene_size_and_determinism():
    a = I.config1_tree()
    b = I.config1_tree()
    assert 19000 <= a.n_leaves <= 21000
    assert np.array_equal(a.child, b.child) and np.array_equal(a.w_hh, b.w_hh)
    assert a.w_sigma.shape == (8, a.n_leaves) and a.w_hh.shape == (3, 14, a.n_leaves)
    assert (a.w_sigma > 0).all()


def test_tile_order_is_a_permutation():
    p = I.tile_order(20, 10)
    assert np.array_equal(np.sort(p), np.arange(200))
    # the first 32 rays form an 8x4 tile
    y, x = np.divmod(p[:32], 20)
    assert x.max() - x.min() == 7 and y.max() - y.min() == 3
