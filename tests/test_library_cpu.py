"""CPU checks of the native library: it builds for sm_103a, loads, and
exports every entry point declared in include/cde.h (no GPU call)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "cde.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cde_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_all_symbols():
    from __graft_entry__ import build
    build()
    from paper_1206_5278_gb300 import cde
    L = cde.lib()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(cde.EXPORTED)
    assert "sm_103a" in cde.cde_version()


def test_last_error_is_empty_string_initially():
    from paper_1206_5278_gb300 import cde
    assert isinstance(cde.last_error(), str)


@pytest.mark.parametrize("n_units,upt,ctas", [(1, 1, 304), (7, 2, 304), (2431, 1, 304), (2432, 1, 304),
                                              (4864, 2, 304), (50000, 2, 304), (12500, 1, 152),
                                              (200000, 2, 304), (123457, 3, 300), (9999, 1, 0), (65, 8, 1)])
def test_tile_partition_covers_every_unit_once_in_order(n_units, upt, ctas):
    """The LOO launches' tile partition (the library's own host/device code):
    every unit in exactly one tile, each tile's units distinct and in a fixed
    order, at most about G log2(n_units / G) + 2G slots when the guided levels
    apply, and the small tiles at the end of the queue no larger than upt."""
    from paper_1206_5278_gb300 import cde
    tiles = cde.cde_loo_tile_partition(n_units, upt, ctas)
    seen = []
    for u0, st, n in tiles:
        assert n >= 1 and st >= 1
        seen.extend(range(u0, u0 + st * n, st))
    assert sorted(seen) == list(range(n_units))
    if ctas > 0 and n_units >= 8 * ctas * upt:
        import math
        assert len(tiles) <= ctas * (math.log2(n_units / ctas) + 3)
    if ctas >= 2:
        # large tiles (stride G) first, in levels of G tiles that shrink along the queue
        big = [t for t in tiles if t[1] == ctas]
        assert len(big) % ctas == 0 and big == tiles[:len(big)]
        sizes = [t[2] for t in big]
        assert sizes == sorted(sizes, reverse=True)
        assert all(t[1] == 1 and t[2] <= upt for t in tiles[len(big):])
    with pytest.raises(cde.CdeError):
        cde.cde_loo_tile_partition(0, upt, ctas)
