"""The server's batch formation (host logic, CPU): shortest remaining work first, an age
limit against starvation, the pair cap and the item cap."""
from types import SimpleNamespace as NS

from paper_2204_03139_gb300.serve import form_batch


def _items(spec):
    """spec: [(name, arrival, [pairs of each item])] -> items in admission order."""
    out = []
    for name, arrival, parts in spec:
        req = NS(name=name, arrival=arrival)
        out += [NS(req=req, pairs=p) for p in parts]
    return out


def names(take):
    return [it.req.name for it in take]


def test_shortest_remaining_work_first():
    items = _items([("long", 0.00, [4, 4, 4, 4]), ("short", 0.01, [1]), ("mid", 0.02, [2, 2])])
    take, pairs = form_batch(items, now=0.05, cap=5, max_items=100, max_wait_s=1.0)
    assert names(take) == ["short", "mid", "mid"] and pairs == 5


def test_requests_past_the_age_limit_go_first():
    items = _items([("long", 0.00, [4, 4, 4]), ("short", 0.50, [1])])
    take, _ = form_batch(items, now=0.60, cap=8, max_items=100, max_wait_s=0.2)
    assert names(take) == ["long", "long"]          # waited 0.6 s > 0.2 s: it goes first
    take, _ = form_batch(items, now=0.10, cap=8, max_items=100, max_wait_s=0.2)
    assert names(take)[0] == "short"                # not yet old: shortest first


def test_caps_and_the_first_item_always_fits():
    items = _items([("a", 0.0, [10, 10]), ("b", 0.1, [10])])
    take, pairs = form_batch(items, now=0.2, cap=5, max_items=100, max_wait_s=1.0)
    assert len(take) == 1 and pairs == 10           # one item even above the cap
    take, _ = form_batch(items, now=0.2, cap=100, max_items=2, max_wait_s=1.0)
    assert len(take) == 2
    assert form_batch([], now=0.0, cap=1, max_items=1, max_wait_s=1.0) == ([], 0)
