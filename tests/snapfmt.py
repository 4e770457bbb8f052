"""Reader/writer of the version-3 and version-4 snapshot blobs, for building test inputs.

Format (little-endian, no padding): "PICMCSN1" | u32 version | u32 0 | u64 config hash |
u64 step | u64 n[2] | u64 counters[17] | i64 wall_charge | f64 wall_energy[2] | per species:
u32 cell word[n], f64 frac[n], f64 vx[n], f64 vy[n], f64 vz[n], u64 id[n] | u32 CRC-32 (zlib).
The cell word is cell | next << 18, ``next`` the null-collision countdown pair (k | c << 12) of the
particle (0 for species without the test; 0 in a crafted blob means "not drawn": the restore draws
it).  ``parse`` splits the word into "cell" and "next"; ``build`` joins them.
Counters: wall_hits[2][2], coll[5], near[2], viol[2], births[2], source_pairs, dropped.
Version 4 (tracked neutrals) adds before the CRC: u64 n_neutral | u64 recycled[2] | u64 lost[2] |
u64 ionized | u64 near | the neutral records as above.

This is input plumbing only: it splices particle arrays into a header taken from an existing
blob and recomputes the checksum.  It holds none of the method's arithmetic.
"""
from __future__ import annotations

import struct
import zlib

import numpy as np

HDR = 8 + 4 + 4 + 8 + 8 + 16 + 17 * 8 + 8 + 16
CELL_BITS = 18
CELL_MASK = (1 << CELL_BITS) - 1


def parse(blob: bytes) -> dict:
    assert blob[:8] == b"PICMCSN1"
    ver, _z, h, step, n0, n1 = struct.unpack_from("<IIQQQQ", blob, 8)
    counters = np.frombuffer(blob, np.uint64, 17, 48).copy()
    wall_charge = struct.unpack_from("<q", blob, 48 + 17 * 8)[0]
    wall_energy = np.frombuffer(blob, np.float64, 2, 48 + 17 * 8 + 8).copy()
    off = HDR

    def records(n, off):
        word = np.frombuffer(blob, np.uint32, n, off).copy(); off += 4 * n
        cell = (word & CELL_MASK).astype(np.int32)
        nxt = word >> CELL_BITS
        frac = np.frombuffer(blob, np.float64, n, off).copy(); off += 8 * n
        v = np.stack([np.frombuffer(blob, np.float64, n, off + 8 * n * k) for k in range(3)], 1)
        off += 24 * n
        ids = np.frombuffer(blob, np.uint64, n, off).copy(); off += 8 * n
        return {"cell": cell, "frac": frac, "v": v.copy(), "id": ids, "next": nxt}, off

    sp = []
    for n in (n0, n1):
        r, off = records(n, off)
        sp.append(r)
    out = {"version": ver, "hash": h, "step": step, "counters": counters,
           "wall_charge": wall_charge, "wall_energy": wall_energy, "species": sp}
    if ver == 4:
        nn = struct.unpack_from("<Q", blob, off)[0]
        out["nt_counters"] = np.frombuffer(blob, np.uint64, 6, off + 8).copy()
        out["neutrals"], off = records(nn, off + 56)
    out["crc"] = struct.unpack_from("<I", blob, off)[0]
    assert off + 4 == len(blob)
    return out


def _put_records(out: bytearray, s: dict) -> None:
    o = np.argsort(np.asarray(s["id"], np.uint64), kind="stable")
    nxt = np.asarray(s.get("next", np.zeros(len(o), np.uint32)), np.uint32)
    out += (np.asarray(s["cell"], np.uint32) | (nxt << CELL_BITS))[o].tobytes()
    out += np.asarray(s["frac"], np.float64)[o].tobytes()
    v = np.asarray(s["v"], np.float64).reshape(-1, 3)[o]
    for k in range(3):
        out += np.ascontiguousarray(v[:, k]).tobytes()
    out += np.asarray(s["id"], np.uint64)[o].tobytes()


def build(d: dict) -> bytes:
    """Inverse of ``parse``; particles are written in ascending id order (canonical)."""
    sp = d["species"]
    ver = 4 if "neutrals" in d else 3
    out = bytearray(b"PICMCSN1")
    out += struct.pack("<IIQQQQ", ver, 0, d["hash"], d["step"], len(sp[0]["id"]), len(sp[1]["id"]))
    out += np.asarray(d["counters"], np.uint64).tobytes()
    out += struct.pack("<q", int(d["wall_charge"]))
    out += np.asarray(d["wall_energy"], np.float64).tobytes()
    for s in sp:
        _put_records(out, s)
    if ver == 4:
        out += struct.pack("<Q", len(d["neutrals"]["id"]))
        out += np.asarray(d.get("nt_counters", np.zeros(6)), np.uint64).tobytes()
        _put_records(out, d["neutrals"])
    out += struct.pack("<I", zlib.crc32(bytes(out)) & 0xFFFFFFFF)
    return bytes(out)


def _records_of(s: dict) -> dict:
    x = np.asarray(s["x"], np.float64)
    cell = np.floor(x).astype(np.int32)
    return {"cell": cell, "frac": x - cell, "v": np.asarray(s["v"], np.float64).reshape(-1, 3),
            "id": np.asarray(s["id"], np.uint64), "next": np.asarray(s.get("next", np.zeros(len(x))), np.uint32)}


def with_particles(blob: bytes, species: list, step: int | None = None, neutrals: dict | None = None) -> bytes:
    """Replace the particles of ``blob``; ``species[s]`` (and ``neutrals``, for a version-4 blob)
    has x (dx units), v (n x 3), id (and optionally next, else 0: drawn by the restore).  Counters
    are cleared."""
    d = parse(blob)
    d["counters"] = np.zeros(17, np.uint64)
    d["wall_charge"] = 0
    d["wall_energy"] = np.zeros(2)
    if step is not None:
        d["step"] = step
    d["species"] = [_records_of(s) for s in species]
    if "neutrals" in d:
        d["nt_counters"] = np.zeros(6, np.uint64)
        d["neutrals"] = _records_of(neutrals if neutrals is not None else
                                    {"x": np.zeros(0), "v": np.zeros((0, 3)), "id": np.zeros(0, np.uint64)})
    return build(d)


def round_to_fp32(blob: bytes) -> bytes:
    """Round positions (within the cell) and velocities to FP32-representable values."""
    d = parse(blob)
    for s in d["species"] + ([d["neutrals"]] if "neutrals" in d else []):
        f32 = s["frac"].astype(np.float32)
        wrap = f32 >= np.float32(1.0)
        f32[wrap] = 0.0
        s["cell"] = s["cell"] + wrap.astype(np.int32)
        s["frac"] = f32.astype(np.float64)
        s["v"] = s["v"].astype(np.float32).astype(np.float64)
    return build(d)


def canonical_particles(blob: bytes):
    """(cell, frac, v, id) per species in id order, as parsed."""
    return parse(blob)["species"]
