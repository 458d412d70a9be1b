"""Host logic of the serving loop (no GPU): the admission rule.

Requests are admitted from the head of the waiting queue, in arrival order,
while the resident set stays within its cell, face and slot bounds; a request
that does not fit blocks the ones behind it (no overtaking, so no starvation)."""
import pytest

from paper_2212_00370_gb300 import build as B
from paper_2212_00370_gb300 import rrmhd


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()


def adm(cells, faces, fc, ff, fs):
    return rrmhd.server_admission(cells, faces, fc, ff, fs)


def test_admits_in_order_while_cells_fit():
    assert adm([100, 200, 300], [101, 201, 301], 300, 10**9, 10) == 2
    assert adm([100, 200, 300], [101, 201, 301], 600, 10**9, 10) == 3
    assert adm([100, 200, 300], [101, 201, 301], 99, 10**9, 10) == 0


def test_head_of_line_blocks():
    # the second request does not fit; the small third one must wait behind it
    assert adm([10, 1000, 10], [11, 1001, 11], 100, 10**9, 10) == 1


def test_faces_and_slots_bound_admission():
    # a 64^2 grid has 2 * 64 * 65 faces
    assert adm([4096, 4096], [8320, 8320], 10**9, 10000, 10) == 1
    assert adm([1] * 10, [2] * 10, 10**9, 10**9, 3) == 3
    assert adm([1] * 10, [2] * 10, 10**9, 10**9, 0) == 0


def test_empty_queue():
    assert adm([], [], 100, 100, 5) == 0
