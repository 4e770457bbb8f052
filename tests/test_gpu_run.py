"""The command-line runner on the GPU: diagnostics lines, checkpoints, and a restart from a
checkpoint that ends where the uninterrupted run ends."""
import json

import pytest

from paper_2606_28534_gb300 import build, pic, run
from paper_2606_28534_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    pic.lib()


def _lines(capsys):
    return [json.loads(x) for x in capsys.readouterr().out.splitlines()]


@pytest.mark.parametrize("name", ["SMALL_C2", "SMALL_C6"])
def test_run_checkpoint_and_restart(tmp_path, capsys, name):
    p = W.variant(getattr(W, name), capacity_factor=2.0, **({"neutral_capacity": 2.0} if name == "SMALL_C6" else {}))
    cfg = tmp_path / "cfg.json"
    run.save_config(p, str(cfg))
    a = tmp_path / "a"
    assert run.main(["--config", str(cfg), "--steps", "20", "--diag-every", "5", "--checkpoint-every", "10",
                     "--out", str(a)]) == 0
    lines = _lines(capsys)
    steps = [d["step"] for d in lines if "step" in d]
    assert steps == [5, 10, 15, 20]
    assert all(("neutrals" in d) == (name == "SMALL_C6") for d in lines if "step" in d)
    assert (a / "checkpoint_00000010.bin").exists() and (a / "fields_final.npz").exists()
    # resume at step 10 for 10 more steps: the same final state as the uninterrupted run
    b = tmp_path / "b"
    assert run.main(["--config", str(a / "config.json"), "--restart", str(a / "checkpoint_00000010.bin"),
                     "--steps", "10", "--diag-every", "0", "--out", str(b)]) == 0
    last = _lines(capsys)
    assert [d["step"] for d in last if "step" in d] == [20]
    assert (b / "checkpoint_00000020.bin").read_bytes() == (a / "checkpoint_00000020.bin").read_bytes()
    # a checkpoint of another configuration is refused
    assert run.main(["--config", "c1", "--restart", str(a / "checkpoint_00000010.bin"), "--steps", "1"]) == 3
