"""The Les Houches Event writer (host only): header and <init> block, events
written by the background thread in the order queued, every number read back
as written (12 significant digits for momenta), the closing tag."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2106_10279_gb300 import api
    return api


def _parse(path):
    text = open(path).read()
    assert text.startswith('<LesHouchesEvents version="3.0">')
    assert text.rstrip().endswith("</LesHouchesEvents>")
    init = text.split("<init>\n")[1].split("</init>")[0].split("\n")
    events = []
    for block in text.split("<event>\n")[1:]:
        lines = block.split("</event>")[0].strip().split("\n")
        head = lines[0].split()
        parts = [l.split() for l in lines[1:]]
        events.append((head, parts))
    return init, events


def test_events_round_trip(api, tmp_path):
    rng = np.random.default_rng(1)
    pdg = [21, 21, 6, -6, 21]
    masses = [0.0, 0.0, 173.0, 173.0, 0.0]
    path = tmp_path / "ev.lhe"
    tags = rng.integers(0, 600, size=(6, 5, 2)).astype(np.int32)
    w = api.LheWriter(path, pdg, masses, xsec=1101.2, xsec_error=0.5, w_max=3.0e-3, scale=173.0,
                      colour_tags=tags)
    batches = [rng.normal(size=(n, 4 + 4 * 5)) for n in (7, 0, 13, 1)]
    for b in batches:
        b[:, 3] = rng.integers(-1, 8, size=b.shape[0])       # flow index; -1 and 6, 7: outside the table
    for b in batches:
        w.write(b)
    assert w.close() == 21
    init, events = _parse(path)
    assert init[0].split()[:2] == ["2212", "2212"]
    assert float(init[1].split()[0]) == pytest.approx(1101.2)
    assert int(init[0].split()[8]) == 3
    rec = np.concatenate(batches)
    assert len(events) == rec.shape[0]
    for r, (head, parts) in zip(rec, events):
        assert int(head[0]) == 5 and float(head[2]) == pytest.approx(r[0], rel=1e-10)
        flow = int(r[3])
        for i, row in enumerate(parts):
            assert int(row[0]) == pdg[i]
            assert int(row[1]) == (-1 if i < 2 else 1)
            want = tuple(tags[flow, i]) if 0 <= flow < tags.shape[0] else (0, 0)
            assert (int(row[4]), int(row[5])) == want
            px, py, pz, e, m = map(float, row[6:11])
            assert np.allclose([e, px, py, pz], r[4 + 4 * i:8 + 4 * i], rtol=1e-11, atol=0)
            assert m == masses[i]


def test_bad_arguments(api, tmp_path):
    from paper_2106_10279_gb300 import _lib as L
    with pytest.raises(L.MfError):
        api.LheWriter(tmp_path / "no_such_dir" / "x.lhe", [21, 21, 6], [0, 0, 173])
    with pytest.raises(L.MfError):
        api.LheWriter(tmp_path / "x.lhe", [21, 21], [0, 0])
