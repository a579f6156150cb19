"""Digest of a run of super values, shared by the script that stores the
oracle's section digests and the GPU test that checks the library against
them: the number of set win bits, the number of set not-lose bits, and the
first 16 hex digits of the SHA-256 of the values' bytes ([n, 8] uint64,
little-endian, in layout order).  No step of the method is here."""
import hashlib

import numpy as np


def digest(values) -> tuple[int, int, str]:
    v = np.ascontiguousarray(np.asarray(values, dtype=np.uint64))
    bits = np.unpackbits(v.view(np.uint8).reshape(len(v), 2, 32), axis=2)
    return (int(bits[:, 0].sum()), int(bits[:, 1].sum()),
            hashlib.sha256(v.astype("<u8").tobytes()).hexdigest()[:16])
