"""The factorisation's task list (host code) keeps the claim-order property
and applies every tile update once: compiled with g++ and run (no GPU)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_task_list_counter_protocol(tmp_path):
    exe = str(tmp_path / "chol_tasks_check")
    subprocess.run(["g++", "-std=c++17", "-O1", "-I",
                    os.path.join(ROOT, "paper_1912_07962_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "chol_tasks_check.cc"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_task_list_check_catches_a_planted_mistake(tmp_path):
    # the checker must reject a list whose first grouped update comes before
    # the panel whose tiles it reads
    exe = str(tmp_path / "chol_tasks_check_planted")
    subprocess.run(["g++", "-std=c++17", "-O1", "-DPLANT_EARLY_UPDATE", "-I",
                    os.path.join(ROOT, "paper_1912_07962_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "chol_tasks_check.cc"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode != 0 and "grouped=1" in out.stdout
