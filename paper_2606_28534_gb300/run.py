"""Command-line runner: one simulation from a JSON configuration, stepped on the GPU through the C
ABI, with diagnostics every k steps (one JSON line each, on stdout) and checkpoints every m steps
(snapshot blobs that `--restart` resumes exactly).

    python -m paper_2606_28534_gb300.run --config c2 --steps 300 --diag-every 10 \\
        --checkpoint-every 100 --out run_c2
    python -m paper_2606_28534_gb300.run --config run_c2/config.json \\
        --restart run_c2/checkpoint_00000200.bin --steps 100 --out run_c2b
    python -m paper_2606_28534_gb300.run --config my_sheath.json --dry-run

`--config` takes a path to a JSON object with `pic_config`'s field names (see `include/pic.h`;
missing fields are 0), or the name of a shipped configuration (`configs/<name>.json`: c1 ... c6,
c3p, c6p, the workloads of `workloads.py`).  `--dry-run` validates the configuration and prints
the device workspace it needs without touching a GPU.  `--write-configs` regenerates the shipped
files from `workloads.py`.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

from . import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
CONFIG_DIR = os.path.join(HERE, "configs")
_PAIRS = ("ppc", "mass", "charge", "T")


def _fields() -> set:
    from .pic import PicConfig

    return {name for name, _ in PicConfig._fields_} - {"abi_version", "reserved"}


def load_config(path_or_name: str) -> dict:
    """A configuration dict from a JSON file, or from a shipped configuration by name."""
    path = path_or_name
    if not os.path.exists(path):
        cand = os.path.join(CONFIG_DIR, path_or_name + ".json")
        if not os.path.exists(cand):
            raise FileNotFoundError(f"no configuration file or shipped configuration named {path_or_name!r}")
        path = cand
    with open(path) as f:
        raw = json.load(f)
    if not isinstance(raw, dict):
        raise ValueError(f"{path}: a configuration is a JSON object")
    unknown = sorted(set(raw) - _fields())
    if unknown:
        raise ValueError(f"{path}: unknown configuration fields {unknown}")
    out = {}
    for k, v in raw.items():
        if k in _PAIRS:
            if not (isinstance(v, list) and len(v) == 2):
                raise ValueError(f"{path}: {k} is a pair [electrons, ions]")
            out[k] = tuple(v)
        else:
            out[k] = v
    return out


def save_config(params: dict, path: str) -> None:
    with open(path, "w") as f:
        json.dump({k: (list(v) if isinstance(v, tuple) else v) for k, v in sorted(params.items())}, f, indent=1)
        f.write("\n")


def write_configs(directory: str = CONFIG_DIR) -> list:
    os.makedirs(directory, exist_ok=True)
    names = []
    for name, params in sorted(W.CONFIGS.items()):
        save_config(params, os.path.join(directory, name + ".json"))
        names.append(name)
    return names


def _emit(obj) -> None:
    sys.stdout.write(json.dumps(obj) + "\n")
    sys.stdout.flush()


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--config", help="JSON file or shipped configuration name")
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--diag-every", type=int, default=10, help="0: only at the end")
    ap.add_argument("--checkpoint-every", type=int, default=0, help="0: only at the end (with --out)")
    ap.add_argument("--out", help="directory for config.json, checkpoints and the final fields")
    ap.add_argument("--restart", help="snapshot blob to resume from (same physics configuration)")
    ap.add_argument("--dry-run", action="store_true", help="validate and size the configuration only")
    ap.add_argument("--write-configs", action="store_true", help="regenerate the shipped configurations")
    a = ap.parse_args(argv)

    if a.write_configs:
        _emit({"wrote": write_configs(), "dir": CONFIG_DIR})
        return 0
    if not a.config:
        ap.error("--config is required")
    if a.steps < 0 or a.diag_every < 0 or a.checkpoint_every < 0:
        ap.error("--steps, --diag-every and --checkpoint-every are >= 0")
    from . import pic

    params = load_config(a.config)
    try:
        ws = pic.workspace_size(params)
    except pic.PicError as e:
        _emit({"error": str(e)})
        return 2
    if a.dry_run:
        _emit({"config": a.config, "valid": True, "workspace_bytes": ws})
        return 0

    sim = pic.Simulation(params)
    if a.out:
        os.makedirs(a.out, exist_ok=True)
        save_config(params, os.path.join(a.out, "config.json"))
    if a.restart:
        with open(a.restart, "rb") as f:
            rc = sim.restore(f.read())
        if rc != 0:
            _emit({"error": f"pic_restore of {a.restart}: {pic.STATUS.get(rc, rc)}"})
            return 3
    neutrals = bool(params.get("neutrals"))

    def report():
        d = sim.diag()
        if neutrals:
            d["neutrals"] = sim.neutral_diag()
        _emit(d)

    def checkpoint(step):
        path = os.path.join(a.out, f"checkpoint_{step:08d}.bin")
        with open(path, "wb") as f:
            f.write(sim.snapshot())
        return path

    start = sim.diag()["step"]
    done = 0
    while done < a.steps:
        k = a.steps - done
        for every in (a.diag_every, a.checkpoint_every):
            if every:
                k = min(k, every - (start + done) % every)
        sim.step(k)
        done += k
        step = start + done
        if a.diag_every and step % a.diag_every == 0:
            report()
        if a.out and a.checkpoint_every and step % a.checkpoint_every == 0:
            checkpoint(step)
    sim.sync()
    if not a.diag_every or (start + done) % a.diag_every:
        report()
    if a.out:
        import numpy as np

        last = checkpoint(start + done)
        f = sim.fields()
        np.savez(os.path.join(a.out, "fields_final.npz"), **f)
        _emit({"checkpoint": last, "fields": os.path.join(a.out, "fields_final.npz")})
    sim.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
