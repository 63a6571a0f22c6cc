"""Shared helpers for the tests: moving packed words between numpy and torch."""
import numpy as np

import synth


def to_dev(arr: np.ndarray):
    import torch
    a = np.ascontiguousarray(arr, dtype=np.uint64)
    return torch.from_numpy(a.view(np.int64)).cuda()


def to_host(t) -> np.ndarray:
    return np.ascontiguousarray(t.cpu().numpy()).view(np.uint64)


def valid_words(arr: np.ndarray, cols: int) -> np.ndarray:
    """The words that carry entries (tail bits of the last word masked)."""
    W = synth.words_for(cols)
    out = np.array(arr[:, :W], dtype=np.uint64, copy=True)
    if W:
        out[:, W - 1] &= synth.tail_mask(cols)
    return out


def assert_same_bits(got: np.ndarray, ref: np.ndarray, cols: int, what: str = ""):
    g = valid_words(got, cols)
    r = valid_words(ref, cols)
    if not np.array_equal(g, r):
        bad = np.argwhere(g != r)
        raise AssertionError("%s: %d words differ, first at %s" % (what, len(bad), bad[:5].tolist()))
    # entries beyond `cols` in the last word must be written as zero
    W = synth.words_for(cols)
    if W and cols % 64:
        assert np.all((got[:, W - 1] & ~synth.tail_mask(cols)) == 0), what + ": tail bits not zero"
