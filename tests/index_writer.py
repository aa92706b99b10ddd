"""Test helper: writes hand-made index files in the serialised HSIG format.

Format: b"UNIFYHSG", u32 version 1, u32 section count, then one 96-byte entry per
section {char name[24]; u32 dtype; u32 ndim; u64 shape[4]; u64 offset; u64 nbytes;
u64 checksum; u64 reserved} and 64-byte aligned payloads. Checksum: FNV-1a 64
over little-endian 8-byte words, the last word zero-padded.
"""
import numpy as np

_CODES = {np.dtype(np.int8): 1, np.dtype(np.uint8): 2, np.dtype(np.int32): 3,
          np.dtype(np.uint32): 4, np.dtype(np.int64): 5, np.dtype(np.float32): 6}
ORDER = ["meta", "vectors", "attr", "level", "upper_base", "seg_bounds", "seg_count", "entry_seg",
         "sorted_ids", "skip_next0", "skip_head", "skip_nextU", "adj0", "gmask0", "adjU", "gmaskU"]


def fnv1a_words(b: bytes) -> int:
    b = b + b"\0" * ((-len(b)) % 8)
    h, p, mask = 0xCBF29CE484222325, 0x100000001B3, (1 << 64) - 1
    for w in np.frombuffer(b, dtype="<u8").tolist():
        h = ((h ^ w) * p) & mask
    return h


def write_index(path, sections: dict, corrupt_section: str = None):
    names = [n for n in ORDER if n in sections] + [n for n in sections if n not in ORDER]
    off = (16 + 96 * len(names) + 63) & ~63
    table, payload, offs = bytearray(), [], []
    for nm in names:
        a = np.ascontiguousarray(sections[nm])
        data = a.tobytes()
        ck = fnv1a_words(data)
        if nm == corrupt_section:
            ck ^= 1
        e = bytearray(96)
        e[:len(nm)] = nm.encode()
        e[24:28] = np.uint32(_CODES[a.dtype]).tobytes()
        e[28:32] = np.uint32(a.ndim).tobytes()
        shp = list(a.shape) + [0] * (4 - a.ndim)
        e[32:64] = np.array(shp, dtype="<u8").tobytes()
        e[64:72] = np.uint64(off).tobytes()
        e[72:80] = np.uint64(len(data)).tobytes()
        e[80:88] = np.uint64(ck).tobytes()
        table += e
        payload.append((off, data))
        off = (off + len(data) + 63) & ~63
    with open(path, "wb") as f:
        f.write(b"UNIFYHSG" + np.uint32(1).tobytes() + np.uint32(len(names)).tobytes() + bytes(table))
        for o, data in payload:
            f.seek(o)
            f.write(data)
    return path


def tiny_index_sections(g: dict) -> dict:
    """Sections for a one-layer index described by a golden JSON dict."""
    n, d, S, M = g["n"], g["d"], g["S"], g["M"]
    W = (S * M + 31) // 32
    x = np.asarray(g["x"], np.float32).reshape(n, d)
    attr = np.asarray(g["attr"], np.int64)
    bounds = np.array([np.iinfo(np.int64).min] + list(g["seg_bounds_inner"]) + [np.iinfo(np.int64).max], np.int64)
    seg = np.searchsorted(bounds[1:S], attr, side="right")
    order = np.lexsort((np.arange(n), attr)).astype(np.int32)
    nxt = np.full(n, -1, np.int32)
    nxt[order[:-1]] = order[1:]
    gm = np.zeros((n, W), np.uint32)
    for v, bits in enumerate(g["gmask0_bits"]):
        for b in bits:
            gm[v, b // 32] |= np.uint32(1 << (b % 32))
    entry_seg = np.array([int(np.flatnonzero(seg == j)[0]) if (seg == j).any() else -1 for j in range(S)], np.int32)
    meta = np.zeros(16, np.int64)
    meta[:10] = [n, d, S, M, 0, g["entry_global"], 0, 0, 0, W]
    return dict(meta=meta, vectors=x, attr=attr, level=np.zeros(n, np.int32),
                upper_base=np.full(n, -1, np.int32), seg_bounds=bounds,
                seg_count=np.bincount(seg, minlength=S).astype(np.int64), entry_seg=entry_seg,
                sorted_ids=order, skip_next0=nxt, skip_head=np.array([order[0]], np.int32),
                skip_nextU=np.full(1, -1, np.int32), adj0=np.asarray(g["adj0"], np.int32).reshape(n, S, M),
                gmask0=gm, adjU=np.full((1, S, M), -1, np.int32), gmaskU=np.zeros((1, W), np.uint32))


def layered_index_sections(g: dict) -> dict:
    """Sections for a multi-layer index described by a golden JSON dict: per-node
    levels, upper-layer rows given as {v, l, adj, bits}, the global entry point and
    per-segment entry points. Upper rows are laid out by id, (v, l) at
    upper_base[v] + l - 1; the level-l skip list links the nodes of level >= l in
    (attribute, id) order."""
    sec = tiny_index_sections(g)
    n, S, M = g["n"], g["S"], g["M"]
    W = (S * M + 31) // 32
    level = np.asarray(g["level"], np.int32)
    L = int(level.max())
    upper_base = np.full(n, -1, np.int32)
    rows = 0
    for v in range(n):
        if level[v] > 0:
            upper_base[v] = rows
            rows += int(level[v])
    adjU = np.full((max(rows, 1), S, M), -1, np.int32)
    gmU = np.zeros((max(rows, 1), W), np.uint32)
    for r in g["upper"]:
        row = upper_base[r["v"]] + r["l"] - 1
        adjU[row] = np.asarray(r["adj"], np.int32)
        for b in r["bits"]:
            gmU[row, b // 32] |= np.uint32(1 << (b % 32))
    order = sec["sorted_ids"]
    head = np.full(L + 1, -1, np.int32)
    head[0] = order[0]
    nextU = np.full(max(rows, 1), -1, np.int32)
    for lv in range(1, L + 1):
        chain = [int(v) for v in order if level[v] >= lv]
        head[lv] = chain[0]
        for a, b in zip(chain[:-1], chain[1:]):
            nextU[upper_base[a] + lv - 1] = b
    meta = sec["meta"].copy()
    meta[4] = L
    meta[5] = g["entry_global"]
    meta[6] = rows
    sec.update(meta=meta, level=level, upper_base=upper_base, skip_head=head, skip_nextU=nextU,
               adjU=adjU, gmaskU=gmU, entry_seg=np.asarray(g["entry_seg"], np.int32))
    return sec
