// Launch-shape autotuner: for each kernel family and problem shape it times
// the candidate kernels / tile shapes once, on the shape's real operator data
// and scratch vectors, and keeps the fastest for the rest of the process
// (the table can be written to and read from a text file).
#pragma once
#include <functional>
#include <string>
#include <vector>

#include "common.cuh"

namespace smg {

struct TuneCandidate {
  int id;             // the kernel family's own code for this choice
  const char* name;   // printable tile / path description
};

// Tuning modes: 0 = off (every shape takes its first candidate, the
// untuned default), 1 = time the candidates the first time a shape is seen.
void tune_set_mode(int mode);
int tune_mode();

// The choice for `key`.  A table entry wins; otherwise, with tuning on and
// `st` not capturing a graph, each candidate runs once untimed and then `nrep`
// times between CUDA events on `st` (run(id) launches it), the fastest is
// recorded (ties: the earlier candidate) and returned; otherwise the first
// candidate.  Candidates must leave every output they write in a state the
// caller does not read (scratch buffers).
int tune_pick(const std::string& key, const std::vector<TuneCandidate>& cands, cudaStream_t st,
              const std::function<void(int)>& run, int nrep = 5);

// Pure selection rule: index of the smallest finite time (ties: the lowest
// index), -1 when none is finite.
int tune_fastest(const std::vector<double>& ms);

// Table as text, one entry per line: key, chosen id, chosen name, then
// "name=ms" for every timed candidate (tab separated).
std::string tune_table_text();
// Reads a table written by tune_table_text (the first two fields of each
// line count); returns the number of entries read, -1 on a malformed line.
int tune_table_load(const std::string& text);
void tune_table_clear();

}  // namespace smg
