"""Reads and writes the network checkpoint format of gp_model_save / gp_model_load on the host (no
GPU): magic "GPMPNN01", uint32 version, uint32 parameter count, int64 Adam step, float32 parameters,
first moments and second moments, and (version 2) a uint64 FNV-1a checksum of every byte between the
magic and the checksum.

  python -m paper_1502_07451_b300.models.checkpoint_format FILE          # check FILE
  python -m paper_1502_07451_b300.models.checkpoint_format FILE --to-v2  # rewrite a version 1 file as version 2
"""
import struct
import sys

import numpy as np

MAGIC = b"GPMPNN01"


def fnv1a64(data: bytes, h: int = 0xCBF29CE484222325) -> int:
    """FNV-1a, 64-bit (Fowler, Noll, Vo), over `data`."""
    prime = 0x100000001B3
    mask = (1 << 64) - 1
    for b in data:
        h = ((h ^ b) * prime) & mask
    return h


def read(path):
    """(version, parameter count, step, params, m, v); raises ValueError on a malformed file."""
    with open(path, "rb") as f:
        d = f.read()
    if d[:8] != MAGIC or len(d) < 24:
        raise ValueError("not a checkpoint")
    ver, npar = struct.unpack_from("<II", d, 8)
    (step,) = struct.unpack_from("<q", d, 16)
    end = 24 + 12 * npar
    if ver not in (1, 2) or len(d) != end + (8 if ver == 2 else 0):
        raise ValueError("bad version or length")
    if ver == 2:
        (want,) = struct.unpack_from("<Q", d, end)
        if fnv1a64(d[8:end]) != want:
            raise ValueError("checksum mismatch")
    arr = np.frombuffer(d, dtype="<f4", count=3 * npar, offset=24)
    return ver, npar, step, arr[:npar], arr[npar:2 * npar], arr[2 * npar:]


def write_v2(path, npar, step, params, m, v):
    body = struct.pack("<IIq", 2, npar, step) + np.concatenate([params, m, v]).astype("<f4").tobytes()
    with open(path, "wb") as f:
        f.write(MAGIC + body + struct.pack("<Q", fnv1a64(body)))


if __name__ == "__main__":
    ver, npar, step, p, m, v = read(sys.argv[1])
    print("version %d, %d parameters, step %d" % (ver, npar, step))
    if "--to-v2" in sys.argv and ver == 1:
        write_v2(sys.argv[1], npar, step, p, m, v)
        print("rewritten as version 2")
