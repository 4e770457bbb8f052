"""The command-line runner's host side: shipped configurations, configuration files and dry runs
(validation and workspace size through the C ABI, no GPU)."""
import json
import os

import pytest

from paper_2606_28534_gb300 import build, pic, run
from paper_2606_28534_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    pic.lib()


@pytest.mark.parametrize("name", sorted(W.CONFIGS))
def test_shipped_configurations_are_the_workloads(name):
    assert run.load_config(name) == W.CONFIGS[name]
    assert run.load_config(os.path.join(run.CONFIG_DIR, name + ".json")) == W.CONFIGS[name]


def test_configuration_files_round_trip_and_are_checked(tmp_path, capsys):
    p = W.variant(W.SMALL_C6, K_iz=0.25)
    f = tmp_path / "mine.json"
    run.save_config(p, str(f))
    assert run.load_config(str(f)) == p
    assert run.main(["--config", str(f), "--dry-run"]) == 0
    out = json.loads(capsys.readouterr().out.splitlines()[-1])
    assert out["valid"] and out["workspace_bytes"] == pic.workspace_size(p)
    bad = tmp_path / "bad.json"
    bad.write_text(json.dumps(dict(json.loads(f.read_text()), not_a_field=1)))
    with pytest.raises(ValueError):
        run.load_config(str(bad))
    bad.write_text(json.dumps(dict(json.loads(f.read_text()), ppc=[3])))
    with pytest.raises(ValueError):
        run.load_config(str(bad))
    invalid = tmp_path / "invalid.json"
    run.save_config(W.variant(p, smooth_passes=9), str(invalid))
    assert run.main(["--config", str(invalid), "--dry-run"]) == 2
    with pytest.raises(FileNotFoundError):
        run.load_config("no_such_configuration")
