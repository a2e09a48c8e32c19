"""Address arithmetic of the on-chip two-row-tile form of the tensor-core kernel, restated from
paper_2205_14741_gb300/csrc/k_ns_tc.cu and checked on the CPU (no GPU needed): the drains cover
the image exactly once, the corner operand Bz and the images fit the shared-memory allocation,
the tensor-memory regions are disjoint, and the conversion passes cover every 32-column chunk
once (including the redistribution of warp 10's chunks in quadrant 2)."""

import itertools

import pytest

KB = 1024
WARPS = 12


def img_offset(r, c, rb_count):
    """Byte offset of element (r, c) in a 64 x 64-box, 128-byte-swizzled image (16-bit values)."""
    rb, rr, cb, cc = r >> 6, r & 63, c >> 6, c & 63
    return (cb * rb_count + rb) * 8192 + rr * 128 + (((cc >> 3) ^ (rr & 7)) << 4) + (cc & 7) * 2


def dyn_smem(nb):
    """Usable dynamic shared memory of the kernel (the allocation minus the 1 KB alignment slack)."""
    k_stages, k_stage = (2, 2 * (128 * 128 + 256 * 128)) if nb == 2 else (4, 1 * (128 * 128 + 256 * 128))
    k_res = (nb + 1) * 9 * 8192 + 8192
    return max(k_stages * k_stage, k_res)


@pytest.mark.parametrize("kpad", [160, 192])
def test_drains_write_every_image_element_once(kpad):
    rb_count = (kpad + 63) >> 6
    img_bytes = rb_count * rb_count * 8192
    written = []
    # drain of tile 0: rows 0 .. 127, every column (16-byte groups of 8 elements)
    for r, c in itertools.product(range(128), range(kpad)):
        written.append(img_offset(r, c, rb_count))
    # the transposed copy: element (c, r) for the columns c >= 128 of rows r < 128
    for r, c in itertools.product(range(128), range(128, kpad)):
        written.append(img_offset(c, r, rb_count))
    # the corner: rows and columns 128 ..
    for r, c in itertools.product(range(128, kpad), range(128, kpad)):
        written.append(img_offset(r, c, rb_count))
    want = {img_offset(r, c, rb_count) for r, c in itertools.product(range(kpad), range(kpad))}
    assert len(written) == len(set(written)) == kpad * kpad
    assert set(written) == want
    assert max(written) + 2 <= img_bytes


@pytest.mark.parametrize("kpad,nb", [(160, 2), (192, 2), (160, 1), (192, 1)])
def test_bz_and_images_fit_the_allocation(kpad, nb):
    rb_count = (kpad + 63) >> 6
    img_bytes = rb_count * rb_count * 8192
    bz_off = nb * img_bytes  # after the hi (and lo) image
    wc = kpad - 128
    offs = [img_offset(r, c, rb_count) for r, c in itertools.product(range(kpad), range(wc))]
    assert 0 <= min(offs) and max(offs) + 2 <= rb_count * 8192  # one 64-column block of kpad K rows
    bz_end = bz_off + nb * rb_count * 8192  # hi, then lo
    # the last row tile's A reads 8 KB past the lo (or hi) image: inside the allocation
    assert max(bz_end, nb * img_bytes + 8192) <= dyn_smem(nb)
    # iteration 0's row-sum scratch (at 160 KB, 5 x 192 floats) lies inside the allocation and is
    # dead before Bz is written (the kernel runs the bound before the conversion passes)
    assert 160 * KB + 5 * 192 * 4 <= dyn_smem(nb)


@pytest.mark.parametrize("kpad", [160, 192])
def test_tensor_memory_regions(kpad):
    wc = kpad - 128
    ta = set(range(0, kpad))
    tb = set(range(kpad, kpad + wc))
    r1 = set(range(kpad + wc, kpad + wc + 128))
    tc = set(range(512 - kpad, 512))
    assert max(max(ta), max(tb), max(r1), max(tc)) < 512
    assert not (ta & tb) and not (ta & tc) and not (tb & tc) and not (ta & r1) and not (tb & r1)
    # R1 (iteration 0 only) may overlap TC only where the kernel has finished reading it
    assert (r1 & tc) == (set() if kpad == 160 else set(range(512 - kpad, kpad + wc + 128)))


@pytest.mark.parametrize("kpad", [160, 192])
def test_conversion_chunks_cover_each_chunk_once(kpad):
    for q in range(4):
        seen = []
        for warp in range(WARPS):
            if warp & 3 != q:
                continue
            part = warp >> 2
            shared2 = q == 2  # the two-tile conversion of tile 0: warp 10 has no chunks
            if shared2 and part == 2:
                continue
            step = 64 if shared2 else 96
            seen += list(range(32 * part, kpad, step))
        assert sorted(seen) == list(range(0, kpad, 32)), (q, sorted(seen))
    # warp 10 (lanes 64 .. 95) has no rows in the corner passes and no chunk in the transposed drain
    part10, q10 = 10 >> 2, 10 & 3
    assert 32 * q10 >= kpad - 128
    assert not list(range(128 + 32 * part10, kpad, 96))
