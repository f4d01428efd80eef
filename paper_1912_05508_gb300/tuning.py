"""Persistent cache of the library's tuned settings (lls_autotune, lls_autotune_batched).

The library keeps the settings it measured in a per-process table (lls_tuning_set /
lls_tuning_get). This module saves them to a JSON file and loads them back into the table, so
a shape is tuned once per GPU model and then reused by every later process. Entries are keyed
by the GPU's name and SM count, the call kind (0 = single solve / QR on m x n, 1 = batched
solve: m = batch size, n = largest n), the shape and the options that change the arithmetic.

Cache file: $LLS_TUNE_CACHE, else ~/.cache/lls_gb300/tuning.json. Writes go to a temporary
file that replaces the cache atomically; an unreadable or corrupted cache counts as empty.
"""
from __future__ import annotations

import json
import os
import tempfile

FIELDS = ("panel_width", "node_mode", "gemm_kernel", "batched_ctas_per_sm", "krylov_ctas", "ms")
OPT_FIELDS = ("gemm_prec", "target", "krylov", "reorth", "panel_leaf")


def cache_path() -> str:
    p = os.environ.get("LLS_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "lls_gb300", "tuning.json")


def make_key(device: str, sms: int, kind: int, m: int, n: int, opts: dict) -> str:
    """The cache key of one setting; `opts` maps OPT_FIELDS to ints."""
    parts = [device.replace("|", "/"), f"sm{int(sms)}", f"kind{int(kind)}", f"{int(m)}x{int(n)}"]
    parts += [f"{f}={int(opts[f])}" for f in OPT_FIELDS]
    return "|".join(parts)


def parse_key(key: str):
    """(device, sms, kind, m, n, opts) of a key written by make_key, or None."""
    parts = key.split("|")
    if len(parts) != 4 + len(OPT_FIELDS):
        return None
    try:
        device = parts[0]
        sms = int(parts[1][2:])
        kind = int(parts[2][4:])
        m, n = (int(v) for v in parts[3].split("x"))
        opts = {}
        for f, p in zip(OPT_FIELDS, parts[4:]):
            name, val = p.split("=")
            if name != f:
                return None
            opts[f] = int(val)
    except ValueError:
        return None
    return device, sms, kind, m, n, opts


def load(path: str | None = None) -> dict:
    """The cache's entries {key: {field: value}}; {} when the file is missing or unreadable."""
    path = path or cache_path()
    try:
        with open(path) as fh:
            data = json.load(fh)
    except (OSError, ValueError):
        return {}
    if not isinstance(data, dict):
        return {}
    out = {}
    for k, v in data.items():
        if isinstance(v, dict) and all(f in v for f in FIELDS) and parse_key(k) is not None:
            out[k] = {f: v[f] for f in FIELDS}
    return out


def save(entries: dict, path: str | None = None) -> None:
    """Write the entries atomically (temporary file in the same folder, then rename)."""
    path = path or cache_path()
    folder = os.path.dirname(os.path.abspath(path))
    os.makedirs(folder, exist_ok=True)
    fd, tmp = tempfile.mkstemp(prefix=".tuning.", suffix=".json", dir=folder)
    try:
        with os.fdopen(fd, "w") as fh:
            json.dump(entries, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        try:
            os.unlink(tmp)
        except OSError:
            pass
        raise


def record(key: str, tuning: dict, path: str | None = None) -> None:
    """Add or replace one entry of the cache file."""
    entries = load(path)
    entries[key] = {f: tuning[f] for f in FIELDS}
    save(entries, path)


def entries_for_device(entries: dict, device: str, sms: int):
    """(kind, m, n, opts, tuning) of every entry measured on this GPU model."""
    out = []
    for k, v in entries.items():
        parsed = parse_key(k)
        if parsed is None:
            continue
        dev, s, kind, m, n, opts = parsed
        if dev == device.replace("|", "/") and s == int(sms):
            out.append((kind, m, n, opts, v))
    return out
