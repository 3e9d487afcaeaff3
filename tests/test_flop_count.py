"""The benchmark's FLOP counts per cell update are the oracle's own arithmetic,
counted by oracle/flop_count.cpp (the unchanged oracle compiled with a
counting number type), so the ALU roofline numerators are reproducible.

* Classic 2D shallow water (the headline): the oracle's step, less the Roe
  averages its transverse solver re-derives (four transverse splits per cell,
  two per interface and direction; the kernel takes them from the normal
  solve).
* SharpClaw 2D Euler, WENO5 characteristic-wise: one L(Q) evaluation (one SSP
  stage), the in-cell Riemann problems included.
* Classic 1D elasticity (f-waves): one step.
* Classic 1D acoustics: one step, less the medium constants the oracle
  re-derives at every interface (c = sqrt(K/rho): a division and a square
  root; Z = rho c and 2 Z, twice: three products).
"""
import json
import os
import subprocess

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def counter(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("flops") / "flop_count")
    subprocess.run(["g++", "-O1", "-std=c++17", "-fpermissive", "-w", "-fopenmp",
                    "-ffp-contract=off", os.path.join(ROOT, "oracle", "flop_count.cpp"), "-o",
                    exe], check=True)

    def run(workload, n):
        env = dict(os.environ, OMP_NUM_THREADS="1")
        out = subprocess.run([exe, workload, str(n)], check=True, capture_output=True, text=True,
                             env=env).stdout
        return json.loads(out)
    return run


def test_sw2d_flops_per_cell(counter):
    r = counter("sw2d", 1024)
    assert r["roe_average"] == 20
    assert abs(r["total"] - 4 * r["roe_average"] - bench.SW2D_FLOPS_PER_CELL) < 0.5, r


def test_euler2d_sharpclaw_flops_per_cell_stage(counter):
    r = counter("euler2d", 1024)
    assert abs(r["total"] - bench.EULER2D_WENO5_FLOPS_PER_CELL_STAGE) < 0.5, r


def test_elasticity1d_flops_per_cell(counter):
    r = counter("elast1d", 1000000)
    assert abs(r["total"] - bench.ELAST1D_FLOPS_PER_CELL) < 0.01, r
    assert abs(r["transcendental"] - 2.0) < 1e-3  # one exp per cell side prepared twice


def test_acoustics1d_flops_per_cell(counter):
    r = counter("acou1d", 1000000)
    assert abs(r["sqrt"] - 1.0) < 1e-4 and abs(r["div"] - 7.0) < 1e-4, r
    assert abs(r["total"] - 5.0 - bench.ACOU1D_FLOPS_PER_CELL) < 0.01, r


def test_counting_type_counts_what_it_should(counter):
    """The counter's own arithmetic on a case with a known count: the 1D
    elasticity step has no branch whose cost depends on the data, so two
    sizes give the same count per cell up to the boundary interfaces."""
    a = counter("elast1d", 10000)
    b = counter("elast1d", 100000)
    assert abs(a["total"] - b["total"]) < 0.02
