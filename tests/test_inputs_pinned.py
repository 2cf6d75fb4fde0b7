"""The seeded input fields are pinned by the SHA-256 of their bytes
(synth/pins.json, written by synth/make_pins.py from synth alone): the host
fields always, the device fields for the environment (torch, CUDA, GPU) that
made them.  A changed generator or library then fails here instead of moving
every parity case and benchmark number silently."""
import pytest

from synth import make_pins


def test_host_fields_match_their_pins():
    pins = make_pins.load()["host"]
    fields = make_pins.host_fields()
    assert set(pins) == set(fields)
    for name, make in fields.items():
        assert make_pins.sha256_of(make()) == pins[name], name


@pytest.mark.gpu
def test_device_fields_match_their_pins_in_this_environment():
    torch = pytest.importorskip("torch")
    env = make_pins.environment_key()
    pins = make_pins.load()["device"].get(env)
    if pins is None:
        pytest.skip(f"no device pins for '{env}' (pinned: {sorted(make_pins.load()['device'])})")
    fields = make_pins.device_fields()
    assert set(pins) == set(fields)
    for name, make in fields.items():
        t = make()
        assert make_pins.sha256_of(t) == pins[name], name
        del t
        torch.cuda.empty_cache()
