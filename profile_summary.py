"""Summarise ncu output into the short text files kept under profiles/.

    python profile_summary.py launches <launches.csv> <title> <command>
    python profile_summary.py capture <report.ncu-rep> <title> <command>
    python profile_summary.py traffic <report.ncu-rep> <precision>
    python profile_summary.py mix <report.ncu-rep> <title> <command> <particles>

`launches`: per kernel, the launch count, total time and share of a
`--metrics gpu__time_duration.sum` launch list (cold-cache, serialised: compare shares).
`capture`: the key counters of a `--set full` capture.  `traffic`: writes the DRAM bytes
per launch of pass_a / pass_b into profiles/traffic.json, keyed by the kernels' source hash
(the benchmark reports it only while the sources are unchanged).  `mix`: the instruction
classes of a capture of the op-class counters, per particle (thread instructions / particles).
"""
from __future__ import annotations

import csv
import io
import json
import os
import re
import subprocess
import sys
from collections import defaultdict

ROOT = os.path.dirname(os.path.abspath(__file__))

KEYS = [
    ("gpu__time_duration.sum", "duration"),
    ("dram__bytes_read.sum", "DRAM read"),
    ("dram__bytes_write.sum", "DRAM write"),
    ("gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed", "DRAM throughput % of peak"),
    ("sm__throughput.avg.pct_of_peak_sustained_elapsed", "SM throughput %"),
    ("sm__issue_active.avg.pct_of_peak_sustained_elapsed", "issue active %"),
    ("sm__warps_active.avg.pct_of_peak_sustained_active", "warps active %"),
    ("smsp__inst_executed.sum", "warp instructions"),
    ("launch__registers_per_thread", "registers/thread"),
    ("launch__grid_size", "grid"),
    ("sm__inst_executed_pipe_fp64.avg.pct_of_peak_sustained_active", "FP64 pipe %"),
    ("sm__inst_executed_pipe_alu.avg.pct_of_peak_sustained_active", "ALU pipe %"),
    ("sm__inst_executed_pipe_fma.avg.pct_of_peak_sustained_active", "FMA pipe %"),
    ("sm__inst_executed_pipe_lsu.avg.pct_of_peak_sustained_active", "LSU pipe %"),
    ("sm__inst_executed_pipe_adu.avg.pct_of_peak_sustained_active", "ADU pipe %"),
    ("smsp__inst_executed_op_branch.sum", "branch instructions"),
    ("l1tex__t_sector_hit_rate.pct", "L1 hit %"),
    ("lts__t_sector_hit_rate.pct", "L2 hit %"),
    ("smsp__average_warps_issue_stalled_long_scoreboard_per_issue_active.ratio", "stall long scoreboard"),
    ("smsp__average_warps_issue_stalled_branch_resolving_per_issue_active.ratio", "stall branch resolving"),
    ("smsp__average_warps_issue_stalled_wait_per_issue_active.ratio", "stall wait"),
    ("smsp__average_warps_issue_stalled_short_scoreboard_per_issue_active.ratio", "stall short scoreboard"),
    ("smsp__average_warps_issue_stalled_not_selected_per_issue_active.ratio", "stall not selected"),
    ("sm__inst_executed_pipe_xu.avg.pct_of_peak_sustained_active", "XU pipe %"),
    ("smsp__sass_thread_inst_executed_op_dfma_pred_on.sum", "FP64 FMA (thread inst)"),
    ("smsp__sass_thread_inst_executed_op_dmul_pred_on.sum", "FP64 MUL (thread inst)"),
    ("smsp__sass_thread_inst_executed_op_dadd_pred_on.sum", "FP64 ADD (thread inst)"),
    ("sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active", "FP64 pipe cycles %"),
    ("smsp__thread_inst_executed.sum", "thread instructions"),
    ("smsp__sass_inst_executed_op_global_red.sum", "global RED instructions (warp)"),
    ("lts__t_requests_op_red.sum", "L2 reduction requests"),
    ("lts__t_sectors_op_red.sum", "L2 reduction sectors"),
    ("lts__t_sectors_op_red.avg.pct_of_peak_sustained_elapsed", "L2 reduction sectors % of peak"),
    ("lts__t_requests_op_atom.sum", "L2 atomic requests"),
    ("lts__throughput.avg.pct_of_peak_sustained_elapsed", "L2 throughput % of peak"),
    ("smsp__sass_inst_executed_op_shared_atom.sum", "shared atomic instructions (warp)"),
    ("smsp__sass_inst_executed_op_shared_ld.sum", "shared load instructions (warp)"),
    ("smsp__sass_inst_executed_op_shared_st.sum", "shared store instructions (warp)"),
    ("l1tex__data_pipe_lsu_wavefronts_mem_shared.sum", "shared wavefronts"),
    ("l1tex__data_pipe_lsu_wavefronts_mem_shared.avg.pct_of_peak_sustained_elapsed", "shared wavefronts % of peak"),
    ("l1tex__data_bank_conflicts_pipe_lsu_mem_shared.sum", "shared bank conflicts"),
    ("l1tex__throughput.avg.pct_of_peak_sustained_elapsed", "L1 throughput % of peak"),
]

# kernels of the time step (the rest of a launch list is set-up and diagnostics)
STEP = ("k_prepass", "k_pass_a", "k_envelope", "k_pass_b", "k_ampere", "k_window", "k_sort_",
        "k_scan_", "k_relocate")


def short(name: str) -> str:
    m = re.search(r"(k_[a-z0-9_]+)(<[^>]*>)?", name)
    return (m.group(1) + (m.group(2) or "")) if m else name[:40]


def launches(path, title, command):
    rows = [r for r in csv.reader(open(path)) if r and not r[0].startswith("==")]
    hdr = rows[0]
    ki, mi, vi = hdr.index("Kernel Name"), hdr.index("Metric Name"), hdr.index("Metric Value")
    unit_i = hdr.index("Metric Unit")
    tot, cnt = defaultdict(float), defaultdict(int)
    for r in rows[1:]:
        if r[mi] != "gpu__time_duration.sum":
            continue
        v = float(r[vi].replace(",", ""))
        scale = {"ns": 1e-3, "us": 1.0, "usecond": 1.0, "nsecond": 1e-3, "ms": 1e3, "msecond": 1e3}.get(r[unit_i], 1.0)
        k = short(r[ki])
        tot[k] += v * scale
        cnt[k] += 1
    allt = sum(tot.values())
    stept = sum(t for k, t in tot.items() if k.startswith(STEP)) or 1.0
    out = [f"# {title}", "", f"Command: `{command}`", "",
           "ncu `--metrics gpu__time_duration.sum --clock-control none` launch list (every launch of",
           "the run; cold-cache and serialised, so shares, not absolute times, carry over).",
           "`step share`: share among the time-step kernels only (set-up and diagnostics excluded).", "",
           "| kernel | launches | total us | share | step share |", "|---|---|---|---|---|"]
    for k, t in sorted(tot.items(), key=lambda kv: -kv[1]):
        ss = f"{t / stept:.3f}" if k.startswith(STEP) else "-"
        out.append(f"| {k} | {cnt[k]} | {t:.1f} | {t / allt:.3f} | {ss} |")
    return "\n".join(out) + "\n"


def raw(rep):
    txt = subprocess.run(["ncu", "-i", rep, "--page", "raw", "--csv"], capture_output=True, text=True).stdout
    rows = list(csv.reader(io.StringIO(txt)))
    return rows[0], rows[1], rows[2:]


def capture(rep, title, command, how="--set full"):
    hdr, units, rows = raw(rep)
    out = [f"# {title}", "", f"Command: `{command}`", "", f"ncu `{how} --clock-control none` capture.", ""]
    names = [short(r[hdr.index("Kernel Name")]) for r in rows]
    out.append("| counter | " + " | ".join(names) + " |")
    out.append("|---|" + "---|" * len(names))
    for key, label in KEYS:
        if key not in hdr:
            continue
        i = hdr.index(key)
        out.append(f"| {label} ({units[i]}) | " + " | ".join(r[i] for r in rows) + " |")
    return "\n".join(out) + "\n"


MIX = [
    ("sm__sass_thread_inst_executed_ops_fadd_fmul_ffma_pred_on.sum", "FP32 add/mul/fma"),
    ("sm__sass_thread_inst_executed_ops_fadd2_fmul2_ffma2_pred_on.sum", "FP32 paired add/mul/fma"),
    ("sm__sass_thread_inst_executed_op_fp32_pred_on.sum", "all FP32"),
    ("sm__sass_thread_inst_executed_op_integer_pred_on.sum", "integer"),
    ("sm__sass_thread_inst_executed_op_bit_pred_on.sum", "bit"),
    ("sm__sass_thread_inst_executed_op_conversion_pred_on.sum", "conversion"),
    ("sm__sass_thread_inst_executed_op_memory_pred_on.sum", "memory"),
    ("sm__sass_thread_inst_executed_op_control_pred_on.sum", "control"),
    ("sm__sass_thread_inst_executed_op_inter_thread_communication_pred_on.sum", "shuffle/vote/reduce"),
    ("sm__sass_thread_inst_executed_op_misc_pred_on.sum", "misc"),
    ("sm__sass_thread_inst_executed_op_uniform_pred_on.sum", "uniform"),
    ("sm__sass_thread_inst_executed_op_fp64_pred_on.sum", "FP64"),
    ("smsp__thread_inst_executed.sum", "all thread instructions"),
    ("smsp__inst_executed.sum", "warp instructions"),
]


def mix(rep, title, command, particles):
    hdr, units, rows = raw(rep)
    n = float(particles)
    names = [short(r[hdr.index("Kernel Name")]) for r in rows]
    out = [f"# {title}", "", f"Command: `{command}`", "",
           "ncu op-class counters (`--metrics <the counters below> --clock-control none`), per particle",
           f"({int(n)} particles per launch): thread instructions whose predicate was on, by class;",
           "the last two rows count every executed instruction.", "",
           "| class | " + " | ".join(names) + " |", "|---|" + "---|" * len(names)]
    for key, label in MIX:
        if key in hdr:
            i = hdr.index(key)
            out.append(f"| {label} | " + " | ".join(f"{float(r[i].replace(',', '')) / n:.2f}" for r in rows) + " |")
    for key, label in (("gpu__time_duration.sum", "duration"),
                       ("smsp__issue_active.avg.pct_of_peak_sustained_active", "issue active %"),
                       ("sm__warps_active.avg.pct_of_peak_sustained_active", "warps active %"),
                       ("launch__registers_per_thread", "registers/thread")):
        if key in hdr:
            i = hdr.index(key)
            out.append(f"| {label} ({units[i]}) | " + " | ".join(r[i] for r in rows) + " |")
    return "\n".join(out) + "\n"


def traffic(rep, prec):
    sys.path.insert(0, ROOT)
    import bench
    hdr, units, rows = raw(rep)
    path = os.path.join(ROOT, "profiles", "traffic.json")
    data = json.load(open(path)) if os.path.exists(path) else {}
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    for r in rows:
        k = short(r[hdr.index("Kernel Name")]).split("<")[0].replace("k_", "")
        rb = float(r[hdr.index("dram__bytes_read.sum")]) * scale[units[hdr.index("dram__bytes_read.sum")]]
        wb = float(r[hdr.index("dram__bytes_write.sum")]) * scale[units[hdr.index("dram__bytes_write.sum")]]
        data[f"{k}:{prec}"] = {"dram_bytes_per_launch": int(rb + wb),
                               "source_sha": bench.source_sha(bench.KERNEL_SOURCES[k])}
    json.dump(data, open(path, "w"), indent=1, sort_keys=True)
    return json.dumps(data, indent=1)


if __name__ == "__main__":
    mode = sys.argv[1]
    if mode == "launches":
        print(launches(*sys.argv[2:5]))
    elif mode == "capture":
        print(capture(*sys.argv[2:5], *(sys.argv[5:6] or ["--set full"])))
    elif mode == "mix":
        print(mix(*sys.argv[2:6]))
    else:
        print(traffic(*sys.argv[2:4]))
