"""The GPU sample stream fed to the oracle's graph pipeline (Sec. 3.1-3.4):
faces, windings and positions from qtv_identify_localize give the same lines
as the oracle's own faces and positions (same types and sample counts on the
analytic cores, lengths within 0.5% and every curve point within 0.25 h of
the oracle's curve: positions that agree to 1e-6 h can still fall on either
side of a box boundary, which moves a sample by a fraction of a box; same
line count and total length within 0.5% on a random tangle), with the Eq. 7
error of the curves reported."""
import numpy as np
import pytest

import oracle
import synth
from oracle import graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def q():
    import paper_1911_12070_gb300 as qtv

    qtv.build()
    h = qtv.Qtv(0)
    yield h
    h.close()


def _gpu_graph(q, host):
    ids, w, xyz, resid, flags = q.identify_localize(torch.from_numpy(host).cuda())
    return graph.face_graph(ids.cpu().numpy().view(np.uint64), w.cpu().numpy(),
                            xyz.cpu().numpy().astype(np.float64), host.shape)


def _oracle_graph(host):
    w, _ = oracle.identify(host)
    ids, wind = oracle.face_list(w)
    loc = oracle.localize(host, ids, wind)
    return graph.face_graph(ids, wind, loc["xyz"], host.shape)


def test_config0_lines_from_gpu_samples(q):
    host = synth.analytic_line_ring()
    a = graph.vectorize(_gpu_graph(q, host), d=4.0)
    b = graph.vectorize(_oracle_graph(host), d=4.0)
    assert [(l["type"], l["closed"], len(l["nodes"])) for l in a["lines"]] == \
           [(l["type"], l["closed"], len(l["nodes"])) for l in b["lines"]]
    for la, lb in zip(a["lines"], b["lines"]):
        assert abs(la["length"] - lb["length"]) < 5e-3 * lb["length"]
        d = np.linalg.norm(la["curve"][:, None, :] - lb["curve"][None, :, :], axis=2)
        assert np.max(d.min(axis=1)) < 0.25
    e = graph.density_error(host, np.vstack([l["curve"] for l in a["lines"]]))
    print(f"config 0 from GPU samples: {len(a['lines'])} lines, Eq. 7 error {e:.2e}")
    assert e < 0.02


def test_random_tangle_lines_from_gpu_samples(q):
    host = synth.random_waves_numpy((48, 48, 48), synth.wave_spec(21, 512))
    a = graph.vectorize(_gpu_graph(q, host), d=4.0)
    b = graph.vectorize(_oracle_graph(host), d=4.0)
    la = sum(l["length"] for l in a["lines"])
    lb = sum(l["length"] for l in b["lines"])
    print(f"48^3 tangle: {len(a['lines'])} lines (oracle {len(b['lines'])}), length {la:.1f} "
          f"(oracle {lb:.1f}), reconnections {a['reconnections']}")
    assert len(a["lines"]) == len(b["lines"])
    assert abs(la - lb) < 5e-3 * lb
