"""Measures the throughput probes of the library on one GPU and prints them
as a Markdown table (the rates the CUDA-core kernels' rooflines use).

    python -m paper_2311_04517_gb300.peaks [--device 0]
"""
import argparse
import subprocess

import torch

from . import hpclust as H


def clocks(device: int) -> str:
    try:
        q = subprocess.run(["nvidia-smi", "-i", str(device), "--query-gpu=name,clocks.sm,clocks.max.sm",
                            "--format=csv,noheader"], capture_output=True, text=True, timeout=20)
        return q.stdout.strip()
    except Exception as e:  # no nvidia-smi: say so
        return f"unavailable ({e.__class__.__name__})"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--device", type=int, default=0)
    a = ap.parse_args()
    torch.cuda.set_device(a.device)
    sms = torch.cuda.get_device_properties(a.device).multi_processor_count
    print(f"device {a.device}: {torch.cuda.get_device_name(a.device)}, {sms} SMs; "
          f"clocks (name, SM, max SM) before: {clocks(a.device)}")
    print()
    print("| probe | rate | per SM per clock at 2070 MHz | one launch |")
    print("|---|---|---|---|")
    for kind, (name, unit) in H.PROBES.items():
        rate, ms = H.hpc_peak_probe(kind, a.device)
        per = rate / sms / 2.07e9
        if unit == "B/s":
            print(f"| {name} | {rate / 1e9:.1f} GB/s | {per:.1f} B | {ms:.3f} ms |")
        else:
            print(f"| {name} | {rate / 1e12:.2f} T{unit} | {per:.1f} | {ms:.3f} ms |")
    print()
    print(f"clocks after: {clocks(a.device)}")


if __name__ == "__main__":
    main()
